// ka_cubic_stream.cuh -- group kernels for three-dimensional lattices (any
// side L with L % 4 == 0, 4 <= L <= 128) stored one word per site and plane
// in split-row order.  The sides 32, 64 and 128 run k_rows and k_pencils;
// every other side runs a general form of the same algorithm (k_rows_any,
// k_pencils_any: partial warps of rows, blocks of fewer pencils with several
// layers per warp, chunks of unequal length along the pencils).  Every side
// has its own instance with the geometry fixed at compile time: the general
// form reading the side at run time ran 1.6 times slower at L = 128 (51.8
// against 31.6 us per word-sweep), and instantiated for L = 128 it is still
// 6 % slower than k_pencils (33.6 us), so the three sides keep theirs.
//
// One launch runs one bond-class group (mu, par) -- the four classes
// c = 4(2 mu + par) + a, a = 0..3 -- on one or more one-word state planes
// (64 replicas per site and plane).  Inside a group only the "active"
// pencils (lines along mu whose perpendicular coordinates sum to par mod 2)
// change, and their perpendicular neighbours lie on pencils of the other
// parity and stay fixed, so each active site's count of occupied
// perpendicular neighbours is computed once per group; along a pencil the
// four classes are the bonds (4k+a, 4k+a+1), run in order (section 2.1
// rules (a)-(c) with a random gate; section 3.2 Table 1).
//
// Storage: every row along x holds its L/2 even-x sites, then its L/2 odd-x
// sites.  For mu = 1, 2 the active sites of a row are then one contiguous
// half-row, so a group reads and writes whole 32-byte sectors; for mu = 0 a
// lane's four consecutive sites are two 16-byte chunks, one in each half.
//
// Data movement: every thread loads what it needs straight from global
// memory (the state of one or two planes stays resident in the L2 across
// sweeps), in whole sectors per warp, with many warps per SM in flight; the
// warps of a CTA touch overlapping neighbour rows at the same time, so the
// L1 serves most repeated neighbour reads.  (Staged variants -- a producer
// filling a ring of shared-memory stages by 16-byte cp.async or by tensor
// copies, with mbarrier hand-off -- were built and measured first: the
// copy engines kept too few bytes in flight per SM for this access pattern
// and ran 2-3 times slower than direct loads.)
//
// Compute: counts of the four perpendicular neighbours as masks
// A = [count <= m-1], B = [count <= m] (bit-sliced over 64 replicas), the
// Philox gate blocks, and the four classes along the pencil.
//
// Gates: the bonds at pencil positions 4k+2b and 4k+2b+1 (classes 4g+2b and
// 4g+2b+1) take the two 64-bit halves of the Philox4x32-10 block at counter
// (sweep, 4g+2b, base site of the first, word); site indices are canonical.
#pragma once

#include "ka_internal.cuh"

namespace ka {
namespace stream {

constexpr int kMaxPlanes = 4;

// Compile-time geometry of side L.
template <int L>
struct Geo {
  static constexpr int Lh = L / 2;
  static constexpr int S = L / 4;                       // lanes per row (mu = 0)
  static constexpr int PW = 32 / S;                     // rows per warp (mu = 0)
  static constexpr int Ty = (8 * PW < L) ? 8 * PW : L;  // mu = 0: y extent of a CTA's block
};

// One state plane of one job of a batch (batched launches: one table entry
// per plane of every job of a side and m).  The job runs sweep t_base + s of
// the round's sweep offset s while that is below t_end; after it idles.
struct StreamUnit {
  uint64_t* n;
  uint64_t* p;
  uint32_t t_base, t_end, word0, pad;
  RoundKeys rk;
};

struct Args {
  uint64_t* n;
  uint64_t* p;
  size_t plane;     // elements per plane
  int nplanes;      // planes of this launch (batched: units)
  int L;            // side
  int mu, par;
  uint32_t t, cls0, word0;  // batched: t = the round's sweep offset
  RoundKeys rk;
  const StreamUnit* units;  // batched launches: the unit table, else null
};

// L = the side (every multiple of 4 up to 128 has its instance); batched
// launches (a.units set) run the B = true instances
template <int L>
cudaError_t launch_l(const Args& a, int m, cudaStream_t st);

#define KA_STREAM_EXTERN(LL) \
  extern template cudaError_t launch_l<LL>(const Args&, int, cudaStream_t);
KA_STREAM_EXTERN(4) KA_STREAM_EXTERN(8) KA_STREAM_EXTERN(12) KA_STREAM_EXTERN(16)
KA_STREAM_EXTERN(20) KA_STREAM_EXTERN(24) KA_STREAM_EXTERN(28) KA_STREAM_EXTERN(32)
KA_STREAM_EXTERN(36) KA_STREAM_EXTERN(40) KA_STREAM_EXTERN(44) KA_STREAM_EXTERN(48)
KA_STREAM_EXTERN(52) KA_STREAM_EXTERN(56) KA_STREAM_EXTERN(60) KA_STREAM_EXTERN(64)
KA_STREAM_EXTERN(68) KA_STREAM_EXTERN(72) KA_STREAM_EXTERN(76) KA_STREAM_EXTERN(80)
KA_STREAM_EXTERN(84) KA_STREAM_EXTERN(88) KA_STREAM_EXTERN(92) KA_STREAM_EXTERN(96)
KA_STREAM_EXTERN(100) KA_STREAM_EXTERN(104) KA_STREAM_EXTERN(108) KA_STREAM_EXTERN(112)
KA_STREAM_EXTERN(116) KA_STREAM_EXTERN(120) KA_STREAM_EXTERN(124) KA_STREAM_EXTERN(128)
#undef KA_STREAM_EXTERN

#ifdef KA_STREAM_INSTANCES
namespace {

__device__ __forceinline__ uint64_t okmask(uint64_t x, uint64_t A, uint64_t B) {
  return (x & A) | (~x & B);
}

// Batched launches: the CTA's unit, copied into (dynamic) shared memory;
// false when the unit idles in this sweep of the round (the whole CTA leaves).
__device__ __forceinline__ bool load_unit(const Args& a, int unit, StreamUnit& su) {
  const uint32_t* src = reinterpret_cast<const uint32_t*>(a.units + unit);
  if (threadIdx.x < sizeof(StreamUnit) / 4) reinterpret_cast<uint32_t*>(&su)[threadIdx.x] = src[threadIdx.x];
  __syncthreads();
  return su.t_base + a.t < su.t_end;
}

// The Philox keys of a launch: its own (single job) or its unit's.
template <bool B>
__device__ __forceinline__ const RoundKeys& keys(const Args& a, const StreamUnit& su) {
  if constexpr (B) return su.rk;
  else return a.rk;
}

__device__ __forceinline__ StreamUnit& unit_smem() {
  extern __shared__ __align__(16) unsigned char ka_stream_dsm[];
  return *reinterpret_cast<StreamUnit*>(ka_stream_dsm);
}

// A = [count <= M-1], B = [count <= M] for the count of four set bits per
// replica (the four perpendicular neighbours)
template <int M>
__device__ __forceinline__ void masks4(uint64_t a, uint64_t b, uint64_t c, uint64_t d, uint64_t& A,
                                       uint64_t& B) {
  const uint64_t o3 = a | b | c;                   // at least one of a, b, c
  const uint64_t m3 = (a & b) | (c & (a | b));     // at least two of a, b, c
  const uint64_t a3 = a & b & c;                   // all three
  const uint64_t at1 = o3 | d, at2 = m3 | (d & o3), at3 = a3 | (d & m3), at4 = a3 & d;
  // [count <= k] = not [count >= k + 1]
  auto le = [&](int k) -> uint64_t {
    return k < 0 ? 0ull : k == 0 ? ~at1 : k == 1 ? ~at2 : k == 2 ? ~at3 : k == 3 ? ~at4 : ~0ull;
  };
  A = le(M - 1);
  B = le(M);
}

// The four classes of the group along one pencil whose 4-site segments are
// held by consecutive lanes (prev / next: the lanes of the neighbouring
// segments, periodic).  nn: the segment's words (updated in place); mA, mB:
// masks of the perpendicular counts; fl: receives the swaps of each site.
__device__ __forceinline__ void run_chain(uint64_t (&nn)[4], const uint64_t (&mA)[4],
                                          const uint64_t (&mB)[4], uint64_t (&fl)[4], uint4 g01,
                                          uint4 g23, int prev, int next) {
  // class 0: bond (s0, s1); s0's other along-neighbour is the previous
  // segment's s3 (at its group-start value), s1's is s2
  {
    const uint64_t left = __shfl_sync(0xffffffffu, nn[3], prev);
    const uint64_t sw =
        (nn[0] ^ nn[1]) & lo64(g01) & okmask(left, mA[0], mB[0]) & okmask(nn[2], mA[1], mB[1]);
    nn[0] ^= sw;
    nn[1] ^= sw;
    fl[0] = sw;
    fl[1] = sw;
  }
  // class 1: bond (s1, s2); other along-neighbours s0 and s3
  {
    const uint64_t sw =
        (nn[1] ^ nn[2]) & hi64(g01) & okmask(nn[0], mA[1], mB[1]) & okmask(nn[3], mA[2], mB[2]);
    nn[1] ^= sw;
    nn[2] ^= sw;
    fl[1] |= sw;
    fl[2] = sw;
  }
  // class 2: bond (s2, s3); s3's other along-neighbour is the next segment's
  // s0, which only class 0 has written so far
  const uint64_t right = __shfl_sync(0xffffffffu, nn[0], next);
  {
    const uint64_t sw =
        (nn[2] ^ nn[3]) & lo64(g23) & okmask(nn[1], mA[2], mB[2]) & okmask(right, mA[3], mB[3]);
    nn[2] ^= sw;
    nn[3] ^= sw;
    fl[2] |= sw;
    fl[3] = sw;
  }
  // class 3: bond (s3, next s0); the owner of the next s0 evaluates that
  // site's condition (its other along-neighbour is its s1) and sends it
  {
    const uint64_t mine = okmask(nn[1], mA[0], mB[0]);
    const uint64_t okn = __shfl_sync(0xffffffffu, mine, next);
    const uint64_t sw = (nn[3] ^ right) & hi64(g23) & okmask(nn[2], mA[3], mB[3]) & okn;
    nn[3] ^= sw;
    fl[3] |= sw;
    const uint64_t in = __shfl_sync(0xffffffffu, sw, prev);
    nn[0] ^= in;
    fl[0] |= in;
  }
}



// mu = 0 without staging: a CTA of eight warps takes the 8 PW active rows of a
// block of Ty consecutive y in the two layers z0, z0 + 1 (z0 even), four
// warps per layer.  Every active row's y and z neighbours are rows of the
// block, of its one-row y margin or of the layers z0 - 1, z0 + 2, which the
// block's warps load at the same time, so most neighbour reads of a row are
// served by the L1 after its first load.  Each lane reads and writes its two
// 16-byte chunks (even and odd sites) of every row it touches: whole sectors.
constexpr int kRowWarps = 8;

template <int L, int M, bool B>
__global__ void __launch_bounds__(32 * kRowWarps) k_rows(const __grid_constant__ Args a) {
  using G = Geo<L>;
  constexpr int S = G::S, PW = G::PW, Ty = G::Ty, Lh = G::Lh;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t b = blockIdx.x;
  constexpr int nyb = L / Ty;
  const int yb = (int)(b % nyb);
  b /= nyb;
  const int zp = (int)(b % (L / 2));
  const int plane = (int)(b / (L / 2));
  StreamUnit& su = unit_smem();  // batched: this CTA's unit (plane = unit index)
  if constexpr (B) {
    if (!load_unit(a, plane, su)) return;
  }
  const uint32_t tt = B ? su.t_base + a.t : a.t;  // sweep
  const int z = 2 * zp + warp / (kRowWarps / 2);
  const int gj = lane / S, seg = lane - gj * S;
  const int prev = gj * S + (seg == 0 ? S - 1 : seg - 1);
  const int next = gj * S + (seg == S - 1 ? 0 : seg + 1);
  const int i = (warp % (kRowWarps / 2)) * PW + gj;  // active row of this layer, 0 .. Ty/2 - 1
  const int y = yb * Ty + 2 * i + ((a.par ^ z) & 1);
  // gate blocks (independent of the state: first)
  const uint32_t site =
      (uint32_t)(4 * seg) + (uint32_t)L * ((uint32_t)y + (uint32_t)L * (uint32_t)z);
  const uint32_t word = B ? su.word0 : a.word0 + (uint32_t)plane;
  const uint4 g01 = philox(make_uint4(tt, a.cls0, site, word), keys<B>(a, su));
  const uint4 g23 = philox(make_uint4(tt, a.cls0 + 2, site + 2, word), keys<B>(a, su));
  asm volatile("griddepcontrol.wait;" ::: "memory");
  uint64_t* n = B ? su.n : a.n + (size_t)plane * a.plane;
  uint64_t* p = B ? su.p : a.p + (size_t)plane * a.plane;
  auto row = [&](int yy, int zz) -> size_t { return ((size_t)zz * L + yy) * (size_t)L; };
  const size_t r0 = row(y, z);
  const ulonglong2* cn = reinterpret_cast<const ulonglong2*>(n);
  const ulonglong2* cp = reinterpret_cast<const ulonglong2*>(p);
  // chunk indices (16 bytes): even sites of the segment at seg, odd ones at Lh / 2 + seg
  const size_t e0 = r0 / 2 + seg, o0 = r0 / 2 + Lh / 2 + seg;
  const size_t nb[4] = {row(y == L - 1 ? 0 : y + 1, z) / 2, row(y == 0 ? L - 1 : y - 1, z) / 2,
                        row(y, z == L - 1 ? 0 : z + 1) / 2, row(y, z == 0 ? L - 1 : z - 1) / 2};
  const ulonglong2 ne = cn[e0], no = cn[o0];
  ulonglong2 q[4][2];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    q[k][0] = __ldg(cn + nb[k] + seg);
    q[k][1] = __ldg(cn + nb[k] + Lh / 2 + seg);
  }
  const ulonglong2 pe = cp[e0], po = cp[o0];
  // sites 4 seg + k: even ones in the first half (k = 0, 2), odd ones in the second
  uint64_t nn[4] = {ne.x, no.x, ne.y, no.y}, mA[4], mB[4], fl[4];
  masks4<M>(q[0][0].x, q[1][0].x, q[2][0].x, q[3][0].x, mA[0], mB[0]);
  masks4<M>(q[0][0].y, q[1][0].y, q[2][0].y, q[3][0].y, mA[2], mB[2]);
  masks4<M>(q[0][1].x, q[1][1].x, q[2][1].x, q[3][1].x, mA[1], mB[1]);
  masks4<M>(q[0][1].y, q[1][1].y, q[2][1].y, q[3][1].y, mA[3], mB[3]);
  run_chain(nn, mA, mB, fl, g01, g23, prev, next);
  ulonglong2* gn = reinterpret_cast<ulonglong2*>(n);
  ulonglong2* gp = reinterpret_cast<ulonglong2*>(p);
  gn[e0] = make_ulonglong2(nn[0], nn[2]);
  gn[o0] = make_ulonglong2(nn[1], nn[3]);
  gp[e0] = make_ulonglong2(pe.x & ~fl[0], pe.y & ~fl[2]);
  gp[o0] = make_ulonglong2(po.x & ~fl[1], po.y & ~fl[3]);
}

template <int L, int M>
cudaError_t launch_rows(const Args& a, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.nplanes * (L / 2) * (L / Geo<L>::Ty)));
  cfg.blockDim = dim3(32 * kRowWarps);
  cfg.dynamicSmemBytes = a.units ? sizeof(StreamUnit) : 0;
  cfg.stream = st;
  // single jobs chain their launches (programmatic dependent launch);
  // batched launches do not (a waiting dependent grid slows the running one)
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = a.units ? 0 : 1;
  return a.units ? cudaLaunchKernelEx(&cfg, k_rows<L, M, true>, a)
                 : cudaLaunchKernelEx(&cfg, k_rows<L, M, false>, a);
}

// mu > 0 without staging: lanes take 32 consecutive pencils of the active
// half-row of one layer s (so every load and store of a warp is whole
// sectors), and each of the CTA's eight warps walks one chunk of Lc = L / 8
// positions along the pencils.  Along a chunk the four classes run as a
// wavefront over its four-site segments: iteration j applies classes 0 and
// 1 to segment j, then classes 2 and 3 to segment j - 1, which reproduces
// the class order (class 0 of segment j reads site 4j - 1 before classes 2
// and 3 change it; class 3 of segment j - 1 changes site 4j after class 1
// has read it).  Where chunks meet, the two sides trade the values through
// shared memory: the first site of every chunk after classes 0 and 1 with
// its rule mask, then the swap of the class-3 bond that crosses.
constexpr int kPencilWarps = 8;

template <int L, int M, int MU, bool B>
__global__ void __launch_bounds__(32 * kPencilWarps) k_pencils(const __grid_constant__ Args a) {
  constexpr int Lh = L / 2;
  constexpr int NP = Lh < 32 ? Lh : 32;  // pencils per warp and layer
  constexpr int PL = 32 / NP;            // layers per warp
  constexpr int Lc = L / kPencilWarps;   // positions per chunk
  constexpr int J = Lc / 4;              // segments per chunk
  static_assert(Lc % 4 == 0, "chunks hold whole segments");
  // rows (t, s) start at (s L + t) L (mu = 1) or (t L + s) L (mu = 2): the
  // word strides of one step along the pencil and across layers
  constexpr size_t TS = (MU == 1) ? (size_t)L : (size_t)L * L;
  constexpr size_t SS = (MU == 1) ? (size_t)L * L : (size_t)L;
  constexpr uint32_t CT = (MU == 1) ? (uint32_t)L : (uint32_t)(L * L);  // canonical site steps
  constexpr uint32_t CS = (MU == 1) ? (uint32_t)(L * L) : (uint32_t)L;
  __shared__ uint64_t xn[kPencilWarps][32], xok[kPencilWarps][32], xsw[kPencilWarps][32];
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int nhb = Lh / NP;
  uint32_t b = blockIdx.x;
  const int hb = (int)(b % nhb);
  b /= nhb;
  const int sgrp = (int)(b % (L / PL));
  const int plane = (int)(b / (L / PL));
  StreamUnit& su = unit_smem();  // batched: this CTA's unit (plane = unit index)
  if constexpr (B) {
    if (!load_unit(a, plane, su)) return;
  }
  const uint32_t tt = B ? su.t_base + a.t : a.t;  // sweep
  const int s = sgrp * PL + lane / NP;
  const int h = hb * NP + lane % NP;
  const int act = (a.par ^ s) & 1, oth = act ^ 1;
  const uint32_t x = 2u * (uint32_t)h + (uint32_t)act;  // canonical x of this lane's pencil
  // x neighbours, in the other half: odd[h - 1], odd[h] (x even) or even[h], even[h + 1] (x odd)
  const int hl = act == 0 ? (h == 0 ? Lh - 1 : h - 1) : h;
  const int hr = act == 0 ? h : (h == Lh - 1 ? 0 : h + 1);
  const int sm = s == 0 ? L - 1 : s - 1, sp = s == L - 1 ? 0 : s + 1;
  const int t0 = warp * Lc;
  // position t0 of this lane's pencil, its x neighbours and its neighbours
  // across the layers (same x: the other half of layers s -/+ 1)
  uint64_t* const n = (B ? su.n : a.n + (size_t)plane * a.plane) + (size_t)t0 * TS;
  uint64_t* const p = (B ? su.p : a.p + (size_t)plane * a.plane) + (size_t)t0 * TS;
  uint64_t* const gn = n + (size_t)s * SS + (size_t)act * Lh + h;
  uint64_t* const gp = p + (size_t)s * SS + (size_t)act * Lh + h;
  const uint64_t* const gl = n + (size_t)s * SS + (size_t)oth * Lh + hl;
  const uint64_t* const gr = n + (size_t)s * SS + (size_t)oth * Lh + hr;
  const uint64_t* const gm = n + (size_t)sm * SS + (size_t)act * Lh + h;
  const uint64_t* const gq = n + (size_t)sp * SS + (size_t)act * Lh + h;
  const uint32_t word = B ? su.word0 : a.word0 + (uint32_t)plane;
  const uint32_t site0 = x + (uint32_t)t0 * CT + (uint32_t)s * CS;  // canonical site of t0
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // the previous chunk's last site at the start of the group
  const uint64_t left0 = (t0 == 0) ? gn[(size_t)(L - 1) * TS] : gn[-(ptrdiff_t)TS];
  uint64_t qn[4], qf[4], qp[4], qA2 = 0, qB2 = 0, qA3 = 0, qB3 = 0;  // segment j - 1
  uint4 qg23 = make_uint4(0, 0, 0, 0);
  uint64_t s0n = 0, s0f = 0, s0p = 0;  // the chunk's first site, stored last
#pragma unroll
  for (int k = 0; k < 4; ++k) qn[k] = qf[k] = qp[k] = 0;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    uint64_t cn[4], cp[4], cA[4], cB[4], cf[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const size_t o = (size_t)(4 * j + k) * TS;
      cn[k] = gn[o];
      cp[k] = gp[o];
      masks4<M>(__ldg(gl + o), __ldg(gr + o), __ldg(gm + o), __ldg(gq + o), cA[k], cB[k]);
    }
    const uint32_t st = site0 + (uint32_t)(4 * j) * CT;
    const uint4 g01 = philox(make_uint4(tt, a.cls0, st, word), keys<B>(a, su));
    const uint4 g23 = philox(make_uint4(tt, a.cls0 + 2, st + 2u * CT, word), keys<B>(a, su));
    // class 0: bond (c0, c1); c0's other along-neighbour is site 4j - 1 at its group-start value
    {
      const uint64_t left = (j == 0) ? left0 : qn[3];
      const uint64_t sw = (cn[0] ^ cn[1]) & lo64(g01) & okmask(left, cA[0], cB[0]) &
                          okmask(cn[2], cA[1], cB[1]);
      cn[0] ^= sw;
      cn[1] ^= sw;
      cf[0] = sw;
      cf[1] = sw;
    }
    // class 1: bond (c1, c2); other along-neighbours c0 and c3
    {
      const uint64_t sw = (cn[1] ^ cn[2]) & hi64(g01) & okmask(cn[0], cA[1], cB[1]) &
                          okmask(cn[3], cA[2], cB[2]);
      cn[1] ^= sw;
      cn[2] ^= sw;
      cf[1] |= sw;
      cf[2] = sw;
    }
    cf[3] = 0;
    if (j == 0) {
      // what the previous chunk's classes 2 and 3 need of this chunk's first site
      xn[warp][lane] = cn[0];
      xok[warp][lane] = okmask(cn[1], cA[0], cB[0]);
    } else {
      // class 2 of segment j - 1: bond (q2, q3); q3's other along-neighbour is c0
      {
        const uint64_t sw = (qn[2] ^ qn[3]) & lo64(qg23) & okmask(qn[1], qA2, qB2) &
                            okmask(cn[0], qA3, qB3);
        qn[2] ^= sw;
        qn[3] ^= sw;
        qf[2] |= sw;
        qf[3] |= sw;
      }
      // class 3 of segment j - 1: bond (q3, c0); c0's other along-neighbour is c1
      {
        const uint64_t sw = (qn[3] ^ cn[0]) & hi64(qg23) & okmask(qn[2], qA3, qB3) &
                            okmask(cn[1], cA[0], cB[0]);
        qn[3] ^= sw;
        qf[3] |= sw;
        cn[0] ^= sw;
        cf[0] |= sw;
      }
      // segment j - 1 is final (its first site waits if it is the chunk's first)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (k == 0 && j == 1) continue;
        const size_t o = (size_t)(4 * (j - 1) + k) * TS;
        gn[o] = qn[k];
        gp[o] = qp[k] & ~qf[k];
      }
    }
    if (j == 0) {
      s0n = cn[0];
      s0f = cf[0];
      s0p = cp[0];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      qn[k] = cn[k];
      qf[k] = cf[k];
      qp[k] = cp[k];
    }
    qA2 = cA[2];
    qB2 = cB[2];
    qA3 = cA[3];
    qB3 = cB[3];
    qg23 = g23;
  }
  __syncthreads();
  // classes 2 and 3 of the last segment, with the next chunk's first site
  {
    const int wn = warp == kPencilWarps - 1 ? 0 : warp + 1;
    const uint64_t nx = xn[wn][lane], okn = xok[wn][lane];
    uint64_t sw = (qn[2] ^ qn[3]) & lo64(qg23) & okmask(qn[1], qA2, qB2) & okmask(nx, qA3, qB3);
    qn[2] ^= sw;
    qn[3] ^= sw;
    qf[2] |= sw;
    qf[3] |= sw;
    sw = (qn[3] ^ nx) & hi64(qg23) & okmask(qn[2], qA3, qB3) & okn;
    qn[3] ^= sw;
    qf[3] |= sw;
    xsw[warp][lane] = sw;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (k == 0 && J == 1) continue;
      const size_t o = (size_t)(4 * (J - 1) + k) * TS;
      gn[o] = qn[k];
      gp[o] = qp[k] & ~qf[k];
    }
  }
  __syncthreads();
  // the chunk's first site, after the previous chunk's class-3 bond
  {
    const uint64_t in = xsw[warp == 0 ? kPencilWarps - 1 : warp - 1][lane];
    gn[0] = s0n ^ in;
    gp[0] = s0p & ~(s0f | in);
  }
}

template <int L, int M>
cudaError_t launch_pencils(const Args& a, cudaStream_t st) {
  constexpr int NP = (L / 2) < 32 ? (L / 2) : 32, PL = 32 / NP;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.nplanes * (L / PL) * ((L / 2) / NP)));
  cfg.blockDim = dim3(32 * kPencilWarps);
  cfg.dynamicSmemBytes = a.units ? sizeof(StreamUnit) : 0;
  cfg.stream = st;
  // single jobs chain their launches (programmatic dependent launch);
  // batched launches do not (a waiting dependent grid slows the running one)
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = a.units ? 0 : 1;
  if (a.units)
    return a.mu == 1 ? cudaLaunchKernelEx(&cfg, k_pencils<L, M, 1, true>, a)
                     : cudaLaunchKernelEx(&cfg, k_pencils<L, M, 2, true>, a);
  return a.mu == 1 ? cudaLaunchKernelEx(&cfg, k_pencils<L, M, 1, false>, a)
                   : cudaLaunchKernelEx(&cfg, k_pencils<L, M, 2, false>, a);
}

// Geometry of the mu = 0 launch: a row of L sites is S = L / 4 segments
// (one per lane), PW = 32 / S rows per warp (lanes beyond PW S idle), and a
// CTA's eight warps take the 4 PW active rows of each of two layers in a
// block of Ty = 8 PW consecutive y (rows past L idle).
struct RowGeo {
  int L, S, PW, Ty, nyb;
  __device__ __host__ __forceinline__ explicit RowGeo(int L_) : L(L_) {
    S = L / 4;
    PW = 32 / S;
    Ty = 8 * PW;
    nyb = (L + Ty - 1) / Ty;
  }
};

// Geometry of the mu > 0 launches: NP pencils per warp and layer (the
// largest power of two up to 32 that divides L / 2, so blocks of pencils
// tile a half-row exactly), PL = 32 / NP layers per warp (layers past L
// idle), NS = L / 4 segments per pencil cut into chunks of J consecutive
// segments, one chunk per warp (CW warps of the eight carry a chunk).
struct PencilGeo {
  int L, Lh, NP, PL, nhb, nsg, NS, J, CW;
  __device__ __host__ __forceinline__ explicit PencilGeo(int L_) : L(L_) {
    Lh = L / 2;
    NP = Lh & -Lh;
    if (NP > 32) NP = 32;
    PL = 32 / NP;
    nhb = Lh / NP;
    nsg = (L + PL - 1) / PL;
    NS = L / 4;
    J = (NS + 7) / 8;
    CW = (NS + J - 1) / J;
  }
};

// General form of k_rows (below): the same work with the geometry of RowGeo.
template <int LT, int M, bool B>
__global__ void __launch_bounds__(32 * kRowWarps) k_rows_any(const __grid_constant__ Args a) {
  const RowGeo G(LT);
  const int L = G.L, S = G.S, PW = G.PW, Ty = G.Ty, nyb = G.nyb, Lh = L / 2;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t b = blockIdx.x;
  const int yb = (int)(b % (uint32_t)nyb);
  b /= (uint32_t)nyb;
  const int zp = (int)(b % (uint32_t)(L / 2));
  const int plane = (int)(b / (uint32_t)(L / 2));
  StreamUnit& su = unit_smem();  // batched: this CTA's unit (plane = unit index)
  if constexpr (B) {
    if (!load_unit(a, plane, su)) return;
  }
  const uint32_t tt = B ? su.t_base + a.t : a.t;  // sweep
  const int z = 2 * zp + warp / (kRowWarps / 2);
  const int gj = lane / S, seg = lane - gj * S;
  const bool in_row = gj < PW;
  const int prev = in_row ? gj * S + (seg == 0 ? S - 1 : seg - 1) : lane;
  const int next = in_row ? gj * S + (seg == S - 1 ? 0 : seg + 1) : lane;
  const int i = (warp % (kRowWarps / 2)) * PW + gj;  // active row of this layer in the block
  const int y = yb * Ty + 2 * i + ((a.par ^ z) & 1);
  // sides whose rows fill whole warps and blocks have no idle lanes
  constexpr bool kExact = 32 % (LT / 4) == 0 && LT % (8 * (32 / (LT / 4))) == 0;
  const bool live = kExact || (in_row && y < L);
  // gate blocks (independent of the state: first)
  const uint32_t site =
      (uint32_t)(4 * seg) + (uint32_t)L * ((uint32_t)y + (uint32_t)L * (uint32_t)z);
  const uint32_t word = B ? su.word0 : a.word0 + (uint32_t)plane;
  const uint4 g01 = philox(make_uint4(tt, a.cls0, site, word), keys<B>(a, su));
  const uint4 g23 = philox(make_uint4(tt, a.cls0 + 2, site + 2, word), keys<B>(a, su));
  asm volatile("griddepcontrol.wait;" ::: "memory");
  uint64_t* n = B ? su.n : a.n + (size_t)plane * a.plane;
  uint64_t* p = B ? su.p : a.p + (size_t)plane * a.plane;
  auto row = [&](int yy, int zz) -> size_t { return ((size_t)zz * L + yy) * (size_t)L; };
  const ulonglong2* cn = reinterpret_cast<const ulonglong2*>(n);
  const ulonglong2* cp = reinterpret_cast<const ulonglong2*>(p);
  const ulonglong2 zero = make_ulonglong2(0ull, 0ull);
  // chunk indices (16 bytes): even sites of the segment at seg, odd ones at Lh / 2 + seg
  size_t e0 = 0, o0 = 0;
  ulonglong2 ne = zero, no = zero, pe = zero, po = zero, q[4][2];
  if (live) {
    const size_t r0 = row(y, z);
    e0 = r0 / 2 + seg;
    o0 = r0 / 2 + Lh / 2 + seg;
    const size_t nb[4] = {row(y == L - 1 ? 0 : y + 1, z) / 2, row(y == 0 ? L - 1 : y - 1, z) / 2,
                          row(y, z == L - 1 ? 0 : z + 1) / 2, row(y, z == 0 ? L - 1 : z - 1) / 2};
    ne = cn[e0];
    no = cn[o0];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      q[k][0] = __ldg(cn + nb[k] + seg);
      q[k][1] = __ldg(cn + nb[k] + Lh / 2 + seg);
    }
    pe = cp[e0];
    po = cp[o0];
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k][0] = q[k][1] = zero;
  }
  // sites 4 seg + k: even ones in the first half (k = 0, 2), odd ones in the second
  uint64_t nn[4] = {ne.x, no.x, ne.y, no.y}, mA[4], mB[4], fl[4];
  masks4<M>(q[0][0].x, q[1][0].x, q[2][0].x, q[3][0].x, mA[0], mB[0]);
  masks4<M>(q[0][0].y, q[1][0].y, q[2][0].y, q[3][0].y, mA[2], mB[2]);
  masks4<M>(q[0][1].x, q[1][1].x, q[2][1].x, q[3][1].x, mA[1], mB[1]);
  masks4<M>(q[0][1].y, q[1][1].y, q[2][1].y, q[3][1].y, mA[3], mB[3]);
  run_chain(nn, mA, mB, fl, g01, g23, prev, next);
  if (live) {
    ulonglong2* gn = reinterpret_cast<ulonglong2*>(n);
    ulonglong2* gp = reinterpret_cast<ulonglong2*>(p);
    gn[e0] = make_ulonglong2(nn[0], nn[2]);
    gn[o0] = make_ulonglong2(nn[1], nn[3]);
    gp[e0] = make_ulonglong2(pe.x & ~fl[0], pe.y & ~fl[2]);
    gp[o0] = make_ulonglong2(po.x & ~fl[1], po.y & ~fl[3]);
  }
}

template <int LT, int M>
cudaError_t launch_rows_any(const Args& a, cudaStream_t st) {
  const RowGeo G(LT);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.nplanes * (G.L / 2) * G.nyb));
  cfg.blockDim = dim3(32 * kRowWarps);
  cfg.dynamicSmemBytes = a.units ? sizeof(StreamUnit) : 0;
  cfg.stream = st;
  // single jobs chain their launches (programmatic dependent launch);
  // batched launches do not (a waiting dependent grid slows the running one)
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = a.units ? 0 : 1;
  return a.units ? cudaLaunchKernelEx(&cfg, k_rows_any<LT, M, true>, a)
                 : cudaLaunchKernelEx(&cfg, k_rows_any<LT, M, false>, a);
}

// General form of k_pencils (below): NP pencils of PL layers per warp, CW
// chunks of J segments along the pencils (the last may be shorter), the
// chunk ring closed over those CW chunks.
template <int LT, int M, int MU, bool B>
__global__ void __launch_bounds__(32 * kPencilWarps) k_pencils_any(const __grid_constant__ Args a) {
  const PencilGeo G(LT);
  const int L = G.L, Lh = G.Lh, NP = G.NP, PL = G.PL, nhb = G.nhb, J = G.J, CW = G.CW;
  // rows (t, s) start at (s L + t) L (mu = 1) or (t L + s) L (mu = 2): the
  // word strides of one step along the pencil and across layers
  const size_t TS = (MU == 1) ? (size_t)L : (size_t)L * L;
  const size_t SS = (MU == 1) ? (size_t)L * L : (size_t)L;
  const uint32_t CT = (MU == 1) ? (uint32_t)L : (uint32_t)(L * L);  // canonical site steps
  const uint32_t CS = (MU == 1) ? (uint32_t)(L * L) : (uint32_t)L;
  __shared__ uint64_t xn[kPencilWarps][32], xok[kPencilWarps][32], xsw[kPencilWarps][32];
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t b = blockIdx.x;
  const int hb = (int)(b % (uint32_t)nhb);
  b /= (uint32_t)nhb;
  const int sgrp = (int)(b % (uint32_t)G.nsg);
  const int plane = (int)(b / (uint32_t)G.nsg);
  StreamUnit& su = unit_smem();  // batched: this CTA's unit (plane = unit index)
  if constexpr (B) {
    if (!load_unit(a, plane, su)) return;
  }
  const uint32_t tt = B ? su.t_base + a.t : a.t;  // sweep
  const int s = sgrp * PL + lane / NP;
  const int h = hb * NP + lane % NP;
  // layers past L (when PL does not divide L) idle
  constexpr int kNP = ((LT / 2) & -(LT / 2)) < 32 ? ((LT / 2) & -(LT / 2)) : 32;
  constexpr bool kFullLayers = LT % (32 / kNP) == 0;
  constexpr bool kFullChunks = (LT / 4) % kPencilWarps == 0;
  const bool live = kFullLayers || s < L;
  // this warp's chunk: segments j0 .. j0 + nseg - 1; warps past CW carry none
  const int j0 = warp * J;
  const int nseg = kFullChunks ? J : (warp < CW ? min(J, G.NS - j0) : 0);
  const int act = (a.par ^ s) & 1, oth = act ^ 1;
  const uint32_t x = 2u * (uint32_t)h + (uint32_t)act;  // canonical x of this lane's pencil
  // x neighbours, in the other half: odd[h - 1], odd[h] (x even) or even[h], even[h + 1] (x odd)
  const int hl = act == 0 ? (h == 0 ? Lh - 1 : h - 1) : h;
  const int hr = act == 0 ? h : (h == Lh - 1 ? 0 : h + 1);
  const int sm = s == 0 ? L - 1 : s - 1, sp = s >= L - 1 ? 0 : s + 1;
  const int t0 = 4 * j0;
  // position t0 of this lane's pencil, its x neighbours and its neighbours
  // across the layers (same x: the other half of layers s -/+ 1)
  uint64_t* const n = (B ? su.n : a.n + (size_t)plane * a.plane) + (size_t)t0 * TS;
  uint64_t* const p = (B ? su.p : a.p + (size_t)plane * a.plane) + (size_t)t0 * TS;
  uint64_t* const gn = n + (size_t)s * SS + (size_t)act * Lh + h;
  uint64_t* const gp = p + (size_t)s * SS + (size_t)act * Lh + h;
  const uint64_t* const gl = n + (size_t)s * SS + (size_t)oth * Lh + hl;
  const uint64_t* const gr = n + (size_t)s * SS + (size_t)oth * Lh + hr;
  const uint64_t* const gm = n + (size_t)sm * SS + (size_t)act * Lh + h;
  const uint64_t* const gq = n + (size_t)sp * SS + (size_t)act * Lh + h;
  const bool mem = (kFullLayers && kFullChunks) || (live && nseg > 0);  // this lane touches memory
  const uint32_t word = B ? su.word0 : a.word0 + (uint32_t)plane;
  const uint32_t site0 = x + (uint32_t)t0 * CT + (uint32_t)s * CS;  // canonical site of t0
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // the previous chunk's last site at the start of the group
  uint64_t left0 = 0;
  if (mem) left0 = (t0 == 0) ? gn[(size_t)(L - 1) * TS] : gn[-(ptrdiff_t)TS];
  uint64_t qn[4], qf[4], qp[4], qA2 = 0, qB2 = 0, qA3 = 0, qB3 = 0;  // segment j - 1
  uint4 qg23 = make_uint4(0, 0, 0, 0);
  uint64_t s0n = 0, s0f = 0, s0p = 0;  // the chunk's first site, stored last
#pragma unroll
  for (int k = 0; k < 4; ++k) qn[k] = qf[k] = qp[k] = 0;
#pragma unroll
  for (int j = 0; j < (LT / 4 + 7) / 8; ++j) {
    if (j >= nseg) break;
    uint64_t cn[4], cp[4], cA[4], cB[4], cf[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const size_t o = (size_t)(4 * j + k) * TS;
      if (mem) {
        cn[k] = gn[o];
        cp[k] = gp[o];
        masks4<M>(__ldg(gl + o), __ldg(gr + o), __ldg(gm + o), __ldg(gq + o), cA[k], cB[k]);
      } else {
        cn[k] = cp[k] = 0;
        masks4<M>(0, 0, 0, 0, cA[k], cB[k]);
      }
    }
    const uint32_t st = site0 + (uint32_t)(4 * j) * CT;
    const uint4 g01 = philox(make_uint4(tt, a.cls0, st, word), keys<B>(a, su));
    const uint4 g23 = philox(make_uint4(tt, a.cls0 + 2, st + 2u * CT, word), keys<B>(a, su));
    // class 0: bond (c0, c1); c0's other along-neighbour is site 4j - 1 at its group-start value
    {
      const uint64_t left = (j == 0) ? left0 : qn[3];
      const uint64_t sw = (cn[0] ^ cn[1]) & lo64(g01) & okmask(left, cA[0], cB[0]) &
                          okmask(cn[2], cA[1], cB[1]);
      cn[0] ^= sw;
      cn[1] ^= sw;
      cf[0] = sw;
      cf[1] = sw;
    }
    // class 1: bond (c1, c2); other along-neighbours c0 and c3
    {
      const uint64_t sw = (cn[1] ^ cn[2]) & hi64(g01) & okmask(cn[0], cA[1], cB[1]) &
                          okmask(cn[3], cA[2], cB[2]);
      cn[1] ^= sw;
      cn[2] ^= sw;
      cf[1] |= sw;
      cf[2] = sw;
    }
    cf[3] = 0;
    if (j == 0) {
      // what the previous chunk's classes 2 and 3 need of this chunk's first site
      xn[warp][lane] = cn[0];
      xok[warp][lane] = okmask(cn[1], cA[0], cB[0]);
    } else {
      // class 2 of segment j - 1: bond (q2, q3); q3's other along-neighbour is c0
      {
        const uint64_t sw = (qn[2] ^ qn[3]) & lo64(qg23) & okmask(qn[1], qA2, qB2) &
                            okmask(cn[0], qA3, qB3);
        qn[2] ^= sw;
        qn[3] ^= sw;
        qf[2] |= sw;
        qf[3] |= sw;
      }
      // class 3 of segment j - 1: bond (q3, c0); c0's other along-neighbour is c1
      {
        const uint64_t sw = (qn[3] ^ cn[0]) & hi64(qg23) & okmask(qn[2], qA3, qB3) &
                            okmask(cn[1], cA[0], cB[0]);
        qn[3] ^= sw;
        qf[3] |= sw;
        cn[0] ^= sw;
        cf[0] |= sw;
      }
      // segment j - 1 is final (its first site waits if it is the chunk's first)
      if (mem) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (k == 0 && j == 1) continue;
          const size_t o = (size_t)(4 * (j - 1) + k) * TS;
          gn[o] = qn[k];
          gp[o] = qp[k] & ~qf[k];
        }
      }
    }
    if (j == 0) {
      s0n = cn[0];
      s0f = cf[0];
      s0p = cp[0];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      qn[k] = cn[k];
      qf[k] = cf[k];
      qp[k] = cp[k];
    }
    qA2 = cA[2];
    qB2 = cB[2];
    qA3 = cA[3];
    qB3 = cB[3];
    qg23 = g23;
  }
  __syncthreads();
  // classes 2 and 3 of the last segment, with the next chunk's first site
  if (nseg > 0) {
    const int wn = warp == CW - 1 ? 0 : warp + 1;
    const uint64_t nx = xn[wn][lane], okn = xok[wn][lane];
    uint64_t sw = (qn[2] ^ qn[3]) & lo64(qg23) & okmask(qn[1], qA2, qB2) & okmask(nx, qA3, qB3);
    qn[2] ^= sw;
    qn[3] ^= sw;
    qf[2] |= sw;
    qf[3] |= sw;
    sw = (qn[3] ^ nx) & hi64(qg23) & okmask(qn[2], qA3, qB3) & okn;
    qn[3] ^= sw;
    qf[3] |= sw;
    xsw[warp][lane] = sw;
    if (mem) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (k == 0 && nseg == 1) continue;
        const size_t o = (size_t)(4 * (nseg - 1) + k) * TS;
        gn[o] = qn[k];
        gp[o] = qp[k] & ~qf[k];
      }
    }
  }
  __syncthreads();
  // the chunk's first site, after the previous chunk's class-3 bond
  if (nseg > 0 && mem) {
    const uint64_t in = xsw[warp == 0 ? CW - 1 : warp - 1][lane];
    gn[0] = s0n ^ in;
    gp[0] = s0p & ~(s0f | in);
  }
}

template <int LT, int M>
cudaError_t launch_pencils_any(const Args& a, cudaStream_t st) {
  const PencilGeo G(LT);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.nplanes * G.nsg * G.nhb));
  cfg.blockDim = dim3(32 * kPencilWarps);
  cfg.dynamicSmemBytes = a.units ? sizeof(StreamUnit) : 0;
  cfg.stream = st;
  // single jobs chain their launches (programmatic dependent launch);
  // batched launches do not (a waiting dependent grid slows the running one)
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = a.units ? 0 : 1;
  if (a.units)
    return a.mu == 1 ? cudaLaunchKernelEx(&cfg, k_pencils_any<LT, M, 1, true>, a)
                     : cudaLaunchKernelEx(&cfg, k_pencils_any<LT, M, 2, true>, a);
  return a.mu == 1 ? cudaLaunchKernelEx(&cfg, k_pencils_any<LT, M, 1, false>, a)
                   : cudaLaunchKernelEx(&cfg, k_pencils_any<LT, M, 2, false>, a);
}

}  // namespace

template <int L>
cudaError_t launch_l(const Args& a, int m, cudaStream_t st) {
#define KA_M_CASES_ANY(FN)                     \
  switch (m < 5 ? m : 5) {                     \
    case 0: return FN<L, 0>(a, st);            \
    case 1: return FN<L, 1>(a, st);            \
    case 2: return FN<L, 2>(a, st);            \
    case 3: return FN<L, 3>(a, st);            \
    case 4: return FN<L, 4>(a, st);            \
    default: return FN<L, 5>(a, st);           \
  }
#define KA_M_CASES(FN)                         \
  switch (m < 5 ? m : 5) {                     \
    case 0: return FN<L, 0>(a, st);            \
    case 1: return FN<L, 1>(a, st);            \
    case 2: return FN<L, 2>(a, st);            \
    case 3: return FN<L, 3>(a, st);            \
    case 4: return FN<L, 4>(a, st);            \
    default: return FN<L, 5>(a, st);           \
  }
  if constexpr (L != 32 && L != 64 && L != 128) {
    if (a.mu == 0) KA_M_CASES_ANY(launch_rows_any)
    KA_M_CASES_ANY(launch_pencils_any)
  } else {
    if (a.mu == 0) KA_M_CASES(launch_rows)
    KA_M_CASES(launch_pencils)
  }
#undef KA_M_CASES
#undef KA_M_CASES_ANY
}
#endif  // KA_STREAM_INSTANCES

}  // namespace stream
}  // namespace ka
