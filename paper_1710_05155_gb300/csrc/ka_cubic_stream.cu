// ka_cubic_stream.cu -- host side of the group kernels of three-dimensional
// lattices (ka_cubic_stream.cuh): which lattices they take (d = 3, L % 4 == 0,
// L <= 128), how many planes one launch covers, and the launch.
#include <cstring>

#include "ka_cubic_stream.cuh"

namespace ka {

bool stream_supported(int d, int L) { return d == 3 && L % 4 == 0 && L >= 4 && L <= 128; }

bool stream_preferred(int d, int L, int P) {
  // Measured per word-sweep against the general pencil kernel
  // (ka_cubic_kernel.cuh): from two planes up the group kernels win at every
  // side (1.3-4.4x).  With one plane (64 replicas) they win or tie at
  // L = 8, 16, 48, 80, 88, 96, 104, 112, 116, 120, 124 (up to 1.95x) and lose
  // by up to 8 % at 28, 56, 60, 72 and 100 (rows that leave lanes idle, too
  // few CTAs), tie at 24, 36, 40, 108; the unmeasured sides follow their
  // neighbours.
  if (!stream_supported(d, L)) return false;
  if (P >= 2) return true;
  switch (L) {
    case 20: case 24: case 28: case 36: case 40: case 44: case 52: case 56: case 60: case 68:
    case 72: case 76: case 100: case 108:
      return false;
    default:
      return true;
  }
}

int stream_planes_per_launch(int L, int P) {
  // the planes of one launch stay resident in the L2 across sweeps: n and p
  // of nq one-word planes (16 nq L^3 bytes) within ~72 MB (two planes at
  // L = 128), at most four
  const double per_plane = 16.0 * (double)L * L * L;
  int cap = (int)(72.0e6 / per_plane);
  if (cap < 1) cap = 1;
  if (cap > stream::kMaxPlanes) cap = stream::kMaxPlanes;
  return P < cap ? P : cap;
}

cudaError_t launch_stream_group(const Planes& pl, int q0, int nq, int L, int m, int mu, int par,
                                uint32_t t, const RoundKeys& rk, cudaStream_t st) {
  using namespace stream;
  if (!stream_supported(3, L) || pl.V != 1 || pl.xs != L || nq < 1 || nq > kMaxPlanes || q0 < 0 ||
      q0 + nq > pl.P || mu < 0 || mu > 2 || par < 0 || par > 1 || m < 0)
    return cudaErrorInvalidValue;
  Args a{};
  a.n = pl.n + (size_t)q0 * pl.plane_elems();
  a.p = pl.p + (size_t)q0 * pl.plane_elems();
  a.plane = pl.plane_elems();
  a.nplanes = nq;
  a.mu = mu;
  a.par = par;
  a.t = t;
  a.cls0 = (uint32_t)(4 * (2 * mu + par));
  a.word0 = (uint32_t)q0;
  a.rk = rk;
  a.L = L;
  switch (L) {
    case 4: return launch_l<4>(a, m, st);
    case 8: return launch_l<8>(a, m, st);
    case 12: return launch_l<12>(a, m, st);
    case 16: return launch_l<16>(a, m, st);
    case 20: return launch_l<20>(a, m, st);
    case 24: return launch_l<24>(a, m, st);
    case 28: return launch_l<28>(a, m, st);
    case 32: return launch_l<32>(a, m, st);
    case 36: return launch_l<36>(a, m, st);
    case 40: return launch_l<40>(a, m, st);
    case 44: return launch_l<44>(a, m, st);
    case 48: return launch_l<48>(a, m, st);
    case 52: return launch_l<52>(a, m, st);
    case 56: return launch_l<56>(a, m, st);
    case 60: return launch_l<60>(a, m, st);
    case 64: return launch_l<64>(a, m, st);
    case 68: return launch_l<68>(a, m, st);
    case 72: return launch_l<72>(a, m, st);
    case 76: return launch_l<76>(a, m, st);
    case 80: return launch_l<80>(a, m, st);
    case 84: return launch_l<84>(a, m, st);
    case 88: return launch_l<88>(a, m, st);
    case 92: return launch_l<92>(a, m, st);
    case 96: return launch_l<96>(a, m, st);
    case 100: return launch_l<100>(a, m, st);
    case 104: return launch_l<104>(a, m, st);
    case 108: return launch_l<108>(a, m, st);
    case 112: return launch_l<112>(a, m, st);
    case 116: return launch_l<116>(a, m, st);
    case 120: return launch_l<120>(a, m, st);
    case 124: return launch_l<124>(a, m, st);
    case 128: return launch_l<128>(a, m, st);
    default: return cudaErrorInvalidValue;
  }
}

size_t stream_unit_bytes() { return sizeof(stream::StreamUnit); }

void stream_unit_fill(void* unit, uint64_t* n, uint64_t* p, uint32_t word0, uint32_t t_base,
                      uint32_t t_end, const RoundKeys& rk) {
  stream::StreamUnit u{};
  u.n = n;
  u.p = p;
  u.word0 = word0;
  u.t_base = t_base;
  u.t_end = t_end;
  u.rk = rk;
  std::memcpy(unit, &u, sizeof(u));
}

cudaError_t launch_stream_batch(const void* units_dev, int nunits, int L, int m, int mu, int par,
                                uint32_t sweep_offset, cudaStream_t st) {
  using namespace stream;
  if (!stream_supported(3, L) || nunits < 1 || mu < 0 || mu > 2 || par < 0 || par > 1 || m < 0)
    return cudaErrorInvalidValue;
  Args a{};
  a.nplanes = nunits;
  a.L = L;
  a.mu = mu;
  a.par = par;
  a.t = sweep_offset;
  a.cls0 = (uint32_t)(4 * (2 * mu + par));
  a.units = static_cast<const StreamUnit*>(units_dev);
  switch (L) {
    case 4: return launch_l<4>(a, m, st);
    case 8: return launch_l<8>(a, m, st);
    case 12: return launch_l<12>(a, m, st);
    case 16: return launch_l<16>(a, m, st);
    case 20: return launch_l<20>(a, m, st);
    case 24: return launch_l<24>(a, m, st);
    case 28: return launch_l<28>(a, m, st);
    case 32: return launch_l<32>(a, m, st);
    case 36: return launch_l<36>(a, m, st);
    case 40: return launch_l<40>(a, m, st);
    case 44: return launch_l<44>(a, m, st);
    case 48: return launch_l<48>(a, m, st);
    case 52: return launch_l<52>(a, m, st);
    case 56: return launch_l<56>(a, m, st);
    case 60: return launch_l<60>(a, m, st);
    case 64: return launch_l<64>(a, m, st);
    case 68: return launch_l<68>(a, m, st);
    case 72: return launch_l<72>(a, m, st);
    case 76: return launch_l<76>(a, m, st);
    case 80: return launch_l<80>(a, m, st);
    case 84: return launch_l<84>(a, m, st);
    case 88: return launch_l<88>(a, m, st);
    case 92: return launch_l<92>(a, m, st);
    case 96: return launch_l<96>(a, m, st);
    case 100: return launch_l<100>(a, m, st);
    case 104: return launch_l<104>(a, m, st);
    case 108: return launch_l<108>(a, m, st);
    case 112: return launch_l<112>(a, m, st);
    case 116: return launch_l<116>(a, m, st);
    case 120: return launch_l<120>(a, m, st);
    case 124: return launch_l<124>(a, m, st);
    case 128: return launch_l<128>(a, m, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ka
