// ka_sweep_cubic.cu -- host launchers of the cubic-lattice group kernel
// (ka_cubic_kernel.cuh): one instance, or a batch of units from a device table.
#include "ka_cubic_kernel.cuh"

namespace ka {
namespace {

using cubic::GroupArgs;

template <bool B>
cudaError_t dispatch(int d, int V, bool x, const GroupArgs& a, const BatchArgs& ba, int m,
                     unsigned blocks, size_t smem, cudaStream_t st) {
  switch (d) {
    case 1: return cubic::launch_d<1, B>(V, x, a, ba, m, blocks, smem, st);
    case 2: return cubic::launch_d<2, B>(V, x, a, ba, m, blocks, smem, st);
    case 3: return cubic::launch_d<3, B>(V, x, a, ba, m, blocks, smem, st);
    case 4: return cubic::launch_d<4, B>(V, x, a, ba, m, blocks, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_cubic_group(const Planes& pl, int q, const CubicShape& s, int mu, int par,
                               uint32_t t, const RoundKeys& rk, cudaStream_t st) {
  const int d = s.d, L = s.L, V = pl.V;
  if ((V != 1 && V != 2 && V != 4) || L % 4 != 0 || L / 4 > 32 || d < 1 || d > 4 || mu < 0 || mu >= d)
    return cudaErrorInvalidValue;
  GroupArgs a;
  a.n = pl.n + (size_t)q * pl.plane_elems();
  a.p = pl.p + (size_t)q * pl.plane_elems();
  a.L = L;
  a.S = L / 4;
  a.PW = 32 / a.S;
  a.mu = mu;
  a.par = par;
  a.st[0] = 1;
  for (int k = 1; k < 4; ++k) a.st[k] = a.st[k - 1] * L;
  int j = 0;
  for (int k = 0; k < d; ++k)
    if (k != mu) a.pd[j++] = k;
  for (; j < 3; ++j) a.pd[j] = 0;
  a.NP = 1;
  for (int k = 0; k < d - 1; ++k) a.NP *= L;
  if (d >= 2) a.NP /= 2;
  const int tp = kCubicWarps / V, win = 2 * tp;
  a.nwin = (L + win - 1) / win;
  // the swizzle permutes slots inside aligned blocks of 16 entries; an odd
  // pencil stride keeps accesses across pencils on distinct banks
  a.PS = ((L + 15) / 16) * 16 + 1;
  // a CTA covers 8 / V pencils; the windows of mu > 0 have 16 / V columns
  a.t = t;
  a.cls0 = (uint32_t)(4 * (2 * mu + par));
  a.word0 = (uint32_t)(q * V);
  a.rk = rk;
  const bool x = (mu == 0) || d == 1;
  unsigned blocks;
  if (x) {
    blocks = (unsigned)((a.NP + tp - 1) / tp);
  } else {
    int64_t tiles = a.nwin;
    for (int k = 0; k < d - 2; ++k) tiles *= L;
    blocks = (unsigned)tiles;
  }
  a.ntiles = blocks;
  const size_t smem = (size_t)2 * (2 + 2 * (d - 1)) * tp * V * a.PS * sizeof(uint64_t);
  BatchArgs none{};
  none.units = nullptr;
  return dispatch<false>(d, V, x, a, none, s.m, blocks, smem, st);
}

cudaError_t launch_cubic_group_batch(CubicUnit* units_dev, const uint32_t* tile_unit, int nunits,
                                     uint32_t ntiles, int PSmax,
                                     int d, int V, int m, int mu, int par, uint32_t sweep_offset,
                                     cudaStream_t st) {
  if (nunits <= 0 || ntiles == 0) return cudaSuccess;
  if ((V != 1 && V != 2 && V != 4) || d < 1 || d > 4 || mu < 0 || mu >= d)
    return cudaErrorInvalidValue;
  BatchArgs ba;
  ba.units = units_dev;
  ba.tile_unit = tile_unit;
  ba.nunits = nunits;
  ba.mu = mu;
  ba.par = par;
  ba.ntiles = ntiles;
  ba.sweep_offset = sweep_offset;
  ba.PSmax = PSmax;
  GroupArgs none{};
  none.ntiles = 0;
  const bool x = (mu == 0) || d == 1;
  const int tp = kCubicWarps / V;
  const size_t smem = (size_t)2 * (2 + 2 * (d - 1)) * tp * V * PSmax * sizeof(uint64_t);
  return dispatch<true>(d, V, x, none, ba, m, ntiles, smem, st);
}

}  // namespace ka
