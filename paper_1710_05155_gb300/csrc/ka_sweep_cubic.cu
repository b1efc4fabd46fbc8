// ka_sweep_cubic.cu -- cubic-lattice sweep kernel (one bond-class group per launch).
//
// A group (mu, par) is the four classes c = 4(2 mu + par) + a, a = 0..3: all
// bonds along direction mu on the pencils (lines along mu) whose
// perpendicular coordinates sum to par mod 2.  Inside a group only those
// pencils are written; their perpendicular neighbours lie on pencils of the
// other parity and stay fixed, so each site's count of occupied
// perpendicular neighbours is computed once per group.  Along a pencil the
// four classes are bonds (4k+a, 4k+a+1); they run in order, in registers.
//
// Thread layout: a pencil of length L is split into S = L/4 segments of four
// sites; one lane owns one segment of one plane (V words per site), and the
// S lanes of a pencil sit in the same warp, so the along-pencil neighbours of
// a segment are exchanged with warp shuffles.  Several pencils share a warp
// when S < 32.
//
// Exchange rule (section 2.1, rules (a)-(c); section 3.2 Table 1 with a
// random gate): on bond (i, j) the replicas with n_i != n_j, gate bit 1,
// at most m occupied among the other z-1 neighbours of i, and at most m among
// those of j, swap n_i and n_j; the swapped sites lose their persistence bit.
// Everything is bit-sliced over 64 replicas per word.
#include "ka_internal.cuh"

namespace ka {
namespace {

struct GroupArgs {
  uint64_t* n;  // plane base
  uint64_t* p;
  int L;
  int S;        // segments per pencil (L / 4)
  int PW;       // pencils per warp
  int par;
  int64_t NP;   // active pencils
  int64_t smu;  // stride of direction mu
  int64_t ps[3];  // strides of the perpendicular directions, ascending
  uint32_t t;
  uint32_t cls0;  // first class id of the group
  uint32_t ctr3;  // Philox counter word c3 for this plane
  uint32_t half;  // V == 1: which 64-bit half of the block this plane uses
  RoundKeys rk;
};

__device__ __forceinline__ uint64_t maj3(uint64_t a, uint64_t b, uint64_t c) {
  return (a & b) | (c & (a | b));
}

// [count <= T] for a bit-sliced 3-bit count (b2 b1 b0); T is a compile-time constant.
template <int T>
__device__ __forceinline__ uint64_t le3(uint64_t b2, uint64_t b1, uint64_t b0) {
  if constexpr (T < 0) {
    return 0ull;
  } else if constexpr (T >= 7) {
    return ~0ull;
  } else {
    const uint64_t g0 = (T & 1) ? 0ull : b0;
    const uint64_t g1 = (T & 2) ? (b1 & g0) : (b1 | g0);
    const uint64_t g2 = (T & 4) ? (b2 & g1) : (b2 | g1);
    return ~g2;  // not (count > T)
  }
}

// Bit-sliced count of K perpendicular neighbour words (K = 0, 2, 4 or 6).
template <int K>
__device__ __forceinline__ void count_perp(const uint64_t* x, uint64_t& b2, uint64_t& b1,
                                           uint64_t& b0) {
  if constexpr (K == 0) {
    b2 = b1 = b0 = 0;
  } else if constexpr (K == 2) {
    b0 = x[0] ^ x[1];
    b1 = x[0] & x[1];
    b2 = 0;
  } else if constexpr (K == 4) {
    const uint64_t s = x[0] ^ x[1] ^ x[2], c = maj3(x[0], x[1], x[2]);
    b0 = s ^ x[3];
    const uint64_t k = s & x[3];
    b1 = c ^ k;
    b2 = c & k;
  } else {
    const uint64_t s1 = x[0] ^ x[1] ^ x[2], c1 = maj3(x[0], x[1], x[2]);
    const uint64_t s2 = x[3] ^ x[4] ^ x[5], c2 = maj3(x[3], x[4], x[5]);
    b0 = s1 ^ s2;
    const uint64_t k = s1 & s2;
    b1 = c1 ^ c2 ^ k;
    b2 = maj3(c1, c2, k);
  }
}

template <int V>
__device__ __forceinline__ void load_w(const uint64_t* base, int64_t i, uint64_t (&o)[V]) {
  if constexpr (V == 2) {
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(base + 2 * i);
    o[0] = v.x;
    o[1] = v.y;
  } else {
    o[0] = base[i];
  }
}

template <int V>
__device__ __forceinline__ void load_ro(const uint64_t* base, int64_t i, uint64_t (&o)[V]) {
  if constexpr (V == 2) {
    const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(base + 2 * i));
    o[0] = v.x;
    o[1] = v.y;
  } else {
    o[0] = __ldg(base + i);
  }
}

template <int V>
__device__ __forceinline__ void store_w(uint64_t* base, int64_t i, const uint64_t (&o)[V]) {
  if constexpr (V == 2) {
    *reinterpret_cast<ulonglong2*>(base + 2 * i) = make_ulonglong2(o[0], o[1]);
  } else {
    base[i] = o[0];
  }
}

template <int V>
__device__ __forceinline__ void gate(const GroupArgs& a, uint32_t cls, uint32_t bond,
                                     uint64_t (&u)[V]) {
  const uint4 b = philox(make_uint4(a.t, cls, bond, a.ctr3), a.rk);
  if constexpr (V == 2) {
    u[0] = lo64(b);
    u[1] = hi64(b);
  } else {
    u[0] = a.half ? hi64(b) : lo64(b);
  }
}

template <int V>
__device__ __forceinline__ void shfl_w(unsigned mask, const uint64_t (&x)[V], int src,
                                       uint64_t (&o)[V]) {
#pragma unroll
  for (int h = 0; h < V; ++h) o[h] = __shfl_sync(mask, x[h], src);
}

template <int D, int V, int M>
__global__ void __launch_bounds__(256) k_cubic_group(const GroupArgs a) {
  constexpr int KP = 2 * (D - 1);  // perpendicular neighbours per site
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int S = a.S;
  const int grp = lane / S;
  const int seg = lane - grp * S;
  const int64_t pencil = gw * a.PW + grp;
  const bool valid = (grp < a.PW) && (pencil < a.NP);
  const unsigned act = __ballot_sync(0xffffffffu, valid);
  if (!valid) return;
  const int prev = grp * S + (seg == 0 ? S - 1 : seg - 1);
  const int next = grp * S + (seg == S - 1 ? 0 : seg + 1);
  const int L = a.L;

  // perpendicular coordinates of the pencil: y[0] runs over the values of
  // the right parity, the others over all of [0, L)
  int64_t base = 0;
  int64_t offp[3] = {0, 0, 0}, offm[3] = {0, 0, 0};
  if constexpr (D >= 2) {
    const int half = L >> 1;
    int64_t rest = pencil / half;
    const int r0 = (int)(pencil - rest * half);
    int y[3] = {0, 0, 0};
    int hi = 0;
#pragma unroll
    for (int k = 1; k < D - 1; ++k) {
      y[k] = (int)(rest % L);
      rest /= L;
      hi += y[k];
    }
    y[0] = 2 * r0 + ((a.par + hi) & 1);
#pragma unroll
    for (int k = 0; k < D - 1; ++k) {
      base += (int64_t)y[k] * a.ps[k];
      offp[k] = (y[k] == L - 1) ? -(int64_t)(L - 1) * a.ps[k] : a.ps[k];
      offm[k] = (y[k] == 0) ? (int64_t)(L - 1) * a.ps[k] : -a.ps[k];
    }
  }
  int64_t site[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) site[k] = base + (int64_t)(4 * seg + k) * a.smu;

  // own words and per-site thresholds from the perpendicular neighbours:
  // A = [c_perp <= m-1], B = [c_perp <= m]; the condition of a site in a bond
  // along mu is then (other along-pencil neighbour occupied) ? A : B
  uint64_t nn[4][V], A[4][V], B[4][V], fl[4][V];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    load_w<V>(a.n, site[k], nn[k]);
    uint64_t x[KP > 0 ? KP : 1][V];
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      const int64_t off = (j & 1) ? offm[j >> 1] : offp[j >> 1];
      load_ro<V>(a.n, site[k] + off, x[j]);
    }
#pragma unroll
    for (int h = 0; h < V; ++h) {
      uint64_t xs[KP > 0 ? KP : 1];
#pragma unroll
      for (int j = 0; j < KP; ++j) xs[j] = x[j][h];
      uint64_t b2, b1, b0;
      count_perp<KP>(xs, b2, b1, b0);
      A[k][h] = le3<M - 1>(b2, b1, b0);
      B[k][h] = le3<M>(b2, b1, b0);
      fl[k][h] = 0;
    }
  }

  const uint32_t cls0 = a.cls0;
  uint64_t u[V], t1[V], t2[V];

  // class a = 0: bond (s0, s1); s0's other along-neighbour is the previous
  // segment's s3 (unchanged so far), s1's is s2
  shfl_w<V>(act, nn[3], prev, t1);
  gate<V>(a, cls0 + 0, (uint32_t)site[0], u);
#pragma unroll
  for (int h = 0; h < V; ++h) {
    const uint64_t ok0 = (t1[h] & A[0][h]) | (~t1[h] & B[0][h]);
    const uint64_t ok1 = (nn[2][h] & A[1][h]) | (~nn[2][h] & B[1][h]);
    const uint64_t sw = (nn[0][h] ^ nn[1][h]) & u[h] & ok0 & ok1;
    nn[0][h] ^= sw;
    nn[1][h] ^= sw;
    fl[0][h] |= sw;
    fl[1][h] |= sw;
  }
  // class a = 1: bond (s1, s2); other along-neighbours s0 and s3
  gate<V>(a, cls0 + 1, (uint32_t)site[1], u);
#pragma unroll
  for (int h = 0; h < V; ++h) {
    const uint64_t ok1 = (nn[0][h] & A[1][h]) | (~nn[0][h] & B[1][h]);
    const uint64_t ok2 = (nn[3][h] & A[2][h]) | (~nn[3][h] & B[2][h]);
    const uint64_t sw = (nn[1][h] ^ nn[2][h]) & u[h] & ok1 & ok2;
    nn[1][h] ^= sw;
    nn[2][h] ^= sw;
    fl[1][h] |= sw;
    fl[2][h] |= sw;
  }
  // class a = 2: bond (s2, s3); s2's other is s1, s3's other is the next
  // segment's s0 (written by class 0 only, so final for this group until class 3)
  shfl_w<V>(act, nn[0], next, t1);
  gate<V>(a, cls0 + 2, (uint32_t)site[2], u);
#pragma unroll
  for (int h = 0; h < V; ++h) {
    const uint64_t ok2 = (nn[1][h] & A[2][h]) | (~nn[1][h] & B[2][h]);
    const uint64_t ok3 = (t1[h] & A[3][h]) | (~t1[h] & B[3][h]);
    const uint64_t sw = (nn[2][h] ^ nn[3][h]) & u[h] & ok2 & ok3;
    nn[2][h] ^= sw;
    nn[3][h] ^= sw;
    fl[2][h] |= sw;
    fl[3][h] |= sw;
  }
  // class a = 3: bond (s3, next s0).  s3's other is s2; next s0's other is
  // next s1.  The owner of next s0 evaluates that site's condition and sends it.
#pragma unroll
  for (int h = 0; h < V; ++h) t2[h] = (nn[1][h] & A[0][h]) | (~nn[1][h] & B[0][h]);
  uint64_t okn[V];
  shfl_w<V>(act, t2, next, okn);
  gate<V>(a, cls0 + 3, (uint32_t)site[3], u);
  uint64_t swo[V];
#pragma unroll
  for (int h = 0; h < V; ++h) {
    const uint64_t ok3 = (nn[2][h] & A[3][h]) | (~nn[2][h] & B[3][h]);
    swo[h] = (nn[3][h] ^ t1[h]) & u[h] & ok3 & okn[h];
    nn[3][h] ^= swo[h];
    fl[3][h] |= swo[h];
  }
  uint64_t swi[V];
  shfl_w<V>(act, swo, prev, swi);
#pragma unroll
  for (int h = 0; h < V; ++h) {
    nn[0][h] ^= swi[h];
    fl[0][h] |= swi[h];
  }

#pragma unroll
  for (int k = 0; k < 4; ++k) {
    store_w<V>(a.n, site[k], nn[k]);
    uint64_t pk[V];
    load_w<V>(a.p, site[k], pk);
#pragma unroll
    for (int h = 0; h < V; ++h) pk[h] &= ~fl[k][h];
    store_w<V>(a.p, site[k], pk);
  }
}

template <int D, int V>
cudaError_t launch_dv(const GroupArgs& a, int m, int64_t blocks, cudaStream_t st) {
  constexpr int Z = 2 * D;
  const int mm = m < Z - 1 ? m : Z - 1;
  dim3 grid((unsigned)blocks), block(256);
  switch (mm) {
#define KA_CASE(MM)                                              \
  case MM:                                                       \
    if constexpr (MM <= Z - 1) {                                 \
      k_cubic_group<D, V, MM><<<grid, block, 0, st>>>(a);        \
      return cudaGetLastError();                                 \
    }                                                            \
    break;
    KA_CASE(0)
    KA_CASE(1)
    KA_CASE(2)
    KA_CASE(3)
    KA_CASE(4)
    KA_CASE(5)
    KA_CASE(6)
    KA_CASE(7)
#undef KA_CASE
    default:
      break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_cubic_group(const Planes& pl, int q, const CubicShape& s, int mu, int par,
                               uint32_t t, const RoundKeys& rk, cudaStream_t st) {
  const int d = s.d, L = s.L;
  if (L % 4 != 0 || L / 4 > 32 || d < 1 || d > 4) return cudaErrorInvalidValue;
  GroupArgs a;
  a.n = pl.n + (size_t)q * pl.plane_elems();
  a.p = pl.p + (size_t)q * pl.plane_elems();
  a.L = L;
  a.S = L / 4;
  a.PW = 32 / a.S;
  a.par = par;
  int64_t stride[4] = {1, 1, 1, 1};
  for (int k = 1; k < 4; ++k) stride[k] = stride[k - 1] * L;
  a.smu = stride[mu];
  int j = 0;
  for (int k = 0; k < d; ++k)
    if (k != mu) a.ps[j++] = stride[k];
  for (; j < 3; ++j) a.ps[j] = 0;
  a.NP = 1;
  for (int k = 0; k < d - 1; ++k) a.NP *= L;
  if (d >= 2) a.NP /= 2;
  a.t = t;
  a.cls0 = (uint32_t)(4 * (2 * mu + par));
  if (pl.V == 2) {
    a.ctr3 = (uint32_t)q;
    a.half = 0;
  } else {
    a.ctr3 = (uint32_t)(q >> 1);
    a.half = (uint32_t)(q & 1);
  }
  a.rk = rk;
  const int64_t warps = (a.NP + a.PW - 1) / a.PW;
  const int64_t blocks = (warps * 32 + 255) / 256;
  switch (d * 2 + (pl.V == 2 ? 1 : 0)) {
    case 2: return launch_dv<1, 1>(a, s.m, blocks, st);
    case 3: return launch_dv<1, 2>(a, s.m, blocks, st);
    case 4: return launch_dv<2, 1>(a, s.m, blocks, st);
    case 5: return launch_dv<2, 2>(a, s.m, blocks, st);
    case 6: return launch_dv<3, 1>(a, s.m, blocks, st);
    case 7: return launch_dv<3, 2>(a, s.m, blocks, st);
    case 8: return launch_dv<4, 1>(a, s.m, blocks, st);
    case 9: return launch_dv<4, 2>(a, s.m, blocks, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ka
