// ka_cubic_stream.cu -- host side of the group kernels of three-dimensional
// lattices (ka_cubic_stream.cuh): which lattices they take, how many planes
// one launch covers, and the launch.
#include "ka_cubic_stream.cuh"

namespace ka {

bool stream_supported(int d, int L) { return d == 3 && (L == 32 || L == 64 || L == 128); }

int stream_planes_per_launch(int L, int P) {
  // two one-word planes of an L = 128 lattice (n and p: 64 MiB) stay resident
  // in the L2 across sweeps; smaller lattices take up to four planes at once
  const int cap = (L >= 128) ? 2 : stream::kMaxPlanes;
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
  if (L == 32) return launch_l<32>(a, m, st);
  if (L == 64) return launch_l<64>(a, m, st);
  return launch_l<128>(a, m, st);
}

}  // namespace ka
