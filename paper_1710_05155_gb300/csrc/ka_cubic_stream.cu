// ka_cubic_stream.cu -- host side of the group kernels of three-dimensional
// lattices (ka_cubic_stream.cuh): which lattices they take (d = 3, L % 4 == 0,
// L <= 128), how many planes one launch covers, and the launch.
#include "ka_cubic_stream.cuh"

namespace ka {

bool stream_supported(int d, int L) { return d == 3 && L % 4 == 0 && L >= 4 && L <= 128; }

bool stream_preferred(int d, int L, int P) {
  // Measured per word-sweep against the general pencil kernel
  // (ka_cubic_kernel.cuh): the group kernels win at every side from two
  // planes up (1.1-3.6x) and for one plane from L = 96 up when L % 8 == 0
  // (blocks of at least four pencils: 1.1-1.6x); otherwise one plane gives
  // them too few CTAs (e.g. 100 at L = 80) or half-sector rows (L = 100) and
  // the general kernel is 5-25 % faster.  The fixed sides 32, 64 and 128
  // always take them.
  if (!stream_supported(d, L)) return false;
  return L == 32 || L == 64 || L == 128 || P >= 2 || (L >= 96 && L % 8 == 0);
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
  if (L == 32) return launch_l<32>(a, m, st);
  if (L == 64) return launch_l<64>(a, m, st);
  if (L == 128) return launch_l<128>(a, m, st);
  return launch_l<0>(a, m, st);  // every other side: geometry from the arguments
}

}  // namespace ka
