// ka_internal.cuh -- internal declarations of the GB300 multispin KA library.
//
// Device layout of one state plane set (n, n0, p): P = W / V planes, each
// [N][V] uint64, W = R / 64 words per site.  Word w of site i lives in plane
// w / V at element i * V + w % V.  Cubic lattices on the pencil kernel use
// V = 4 (one 32-byte sector per site) when 4 divides W; otherwise V = 2 for
// even W, else 1.
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ka.h"

#define KA_HD __host__ __device__ __forceinline__

namespace ka {

// A named NVTX range for the lifetime of a scope (API calls show up by name
// in profilers; costs nothing when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};


constexpr uint32_t kTagInit = 0xFFFFFFFFu;   // counter word c1 of the initial-state keys
constexpr uint32_t kTagGraph = 0xFFFFFFFEu;  // counter word c1 of the graph shuffle
constexpr uint32_t kTagLayer = 0xFFFFFFFDu;  // counter word c1 of the layer permutations
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// Round keys of Philox4x32-10 for one seed: rk[2r], rk[2r+1] is the key of
// round r (the key is bumped by the Weyl constants between rounds).
struct RoundKeys {
  uint32_t k[20];
};

inline RoundKeys round_keys(uint64_t seed) {
  RoundKeys rk;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk.k[2 * r] = k0;
    rk.k[2 * r + 1] = k1;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return rk;
}

// Philox4x32-10 block (Salmon et al., SC'11) with precomputed round keys.
KA_HD uint4 philox(uint4 c, const RoundKeys& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // one 32 x 32 -> 64-bit multiply per product (a single wide IMAD on the GPU)
    const uint64_t p0 = (uint64_t)kPhiloxM0 * c.x, p1 = (uint64_t)kPhiloxM1 * c.z;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c = make_uint4(hi1 ^ c.y ^ rk.k[2 * r], lo1, hi0 ^ c.w ^ rk.k[2 * r + 1], lo0);
  }
  return c;
}

KA_HD uint64_t lo64(uint4 b) { return (uint64_t)b.x | ((uint64_t)b.y << 32); }
KA_HD uint64_t hi64(uint4 b) { return (uint64_t)b.z | ((uint64_t)b.w << 32); }

// --------------------------------------------------------------------------
// Host-side topology (built at create, uploaded once)
// --------------------------------------------------------------------------
struct Topology {
  int64_t N = 0;
  int z = 0;
  std::vector<int32_t> nbr;        // [N][z]
  std::vector<int64_t> class_off;  // [nclass + 1]
  std::vector<int32_t> bu, bv;     // bonds grouped by class
  std::vector<int64_t> bid;        // Philox bond id
  int attempts = 0;
  int64_t nclass() const { return (int64_t)class_off.size() - 1; }
};

// Returns "" on success, else an error message.
std::string build_cubic_tables(int d, int L, Topology& t);
std::string build_rrg(int64_t N, int z, uint64_t graph_seed, Topology& t);
std::string build_graph(int64_t N, int z, const int32_t* nbr, Topology& t);
// Storage order of a graph's sites: breadth-first from site 0 (then from the
// lowest unvisited site), neighbours in row order.  perm[i] = position of
// canonical site i, inv[q] = canonical site at position q.
void bfs_order(int64_t N, int z, const int32_t* nbr, std::vector<int32_t>& perm,
               std::vector<int32_t>& inv);
// Device tables in storage positions: the neighbour rows relabelled (slot
// order kept), and every class's bonds relabelled and sorted by their lower
// position, each keeping its canonical bond id.
void relabel_tables(const Topology& t, int z, const std::vector<int32_t>& perm,
                    std::vector<int32_t>& nbr, std::vector<int32_t>& bu, std::vector<int32_t>& bv,
                    std::vector<uint32_t>& bid);
// Neighbour rows [M L^d][2d] of the layered random graph (section 5.2).
std::string build_layered(int d, int L, int M, uint64_t graph_seed, int32_t* nbr);

// --------------------------------------------------------------------------
// Kernel launchers
// --------------------------------------------------------------------------
struct Planes {
  uint64_t* n;
  uint64_t* n0;
  uint64_t* p;
  int64_t N;
  int W;  // words per site (R / 64)
  int V;  // words per site per plane (1, 2 or 4)
  int P;  // planes (W / V)
  int xs; // side L of the split-row site order (below), or 0: sites in index order
  const int32_t* inv = nullptr;  // graphs: canonical site at each storage position (device)
  KA_HD size_t plane_elems() const { return (size_t)N * V; }
};

// Site order of a plane.  Cubic lattices of dimension d >= 2 on the pencil
// kernels store every row along x (L sites, L even) as its L/2 even-x sites
// followed by its L/2 odd-x sites (xs = L), so that the sites a group with
// mu > 0 updates in a row form one contiguous half-row; every other plane
// keeps sites in index order (xs = 0).  Position of canonical site i:
KA_HD int64_t dev_site(int xs, int64_t i) {
  if (!xs) return i;
  const int64_t x = i % xs;
  return i - x + (x & 1) * (xs >> 1) + (x >> 1);
}
// and the canonical site at position q
KA_HD int64_t canon_site(int xs, int64_t q) {
  if (!xs) return q;
  const int64_t r = q % xs, h = xs >> 1;
  return q - r + (r < h ? 2 * r : 2 * (r - h) + 1);
}
// split-row order used by a cubic pencil context of dimension d and side L
KA_HD int split_side(int d, int L) { return d >= 2 ? L : 0; }

// Graphs store sites in breadth-first order (a permutation built at context
// creation, ka_topology.cu), so that sites that are close in the graph share
// 32-byte sectors; inv maps a storage position back to its canonical site.
// Canonical site of storage position q in either order (device code):
KA_HD int64_t canon_pos(const int32_t* inv, int xs, int64_t q) {
  return inv ? (int64_t)inv[q] : canon_site(xs, q);
}

// Warps per CTA of the cubic pencil kernel: a tile holds kCubicWarps / V
// active pencils (one warp per pencil-word in the compute phase).
constexpr int kCubicWarps = 8;

struct CubicShape {
  int d, L, m;
};

// One work unit of a batched launch: one state plane of one instance.  Its
// sweep counter t_base lives in device memory; a launch runs sweep
// t_base + sweep offset of every unit whose counter is still below t_end.
struct CubicUnit {
  uint64_t* n;
  uint64_t* p;
  int d, L;
  uint32_t word0;
  uint32_t tile0[2];  // first global tile of this unit: [0] mu = 0, [1] mu > 0
  uint32_t t_base, t_end;
  RoundKeys rk;
};

// Launch-wide arguments of a batched group launch.
struct BatchArgs {
  CubicUnit* units;
  const uint32_t* tile_unit;  // the unit owning each global tile of this launch
  int nunits;
  int mu, par;
  uint32_t ntiles;  // all tiles of all units for this mu
  uint32_t sweep_offset;
  int PSmax;        // largest pencil stride (shared-memory sizing)
};

// Group (mu, par) of sweep t_base + sweep_offset for every unit of a batch
// (all units share d, V and m); ntiles = sum of the units' tiles for this mu,
// tile_unit[g] = the unit owning global tile g.
cudaError_t launch_cubic_group_batch(CubicUnit* units_dev, const uint32_t* tile_unit, int nunits,
                                     uint32_t ntiles, int PSmax,
                                     int d, int V, int m, int mu, int par, uint32_t sweep_offset,
                                     cudaStream_t st);

// One group (mu, par) of four classes on plane q, sweep index t.
cudaError_t launch_cubic_group(const Planes& pl, int q, const CubicShape& s, int mu, int par,
                               uint32_t t, const RoundKeys& rk, cudaStream_t st);

struct GraphDev {
  const int32_t* nbr;  // [N][z]
  const int32_t* bu;
  const int32_t* bv;
  const uint32_t* bid;
  const int32_t* perm;  // graphs: storage position of every canonical site (null: identity)
  int z, m;
  int cubic_L;  // > 0: the bonds are those of a cubic lattice of this side (its gate stream)
};
// Class c (bonds [off, off + count) of the class-ordered bond arrays), all planes.
cudaError_t launch_graph_class(const Planes& pl, const GraphDev& g, int64_t off, int64_t count,
                               uint32_t cls, uint32_t t, const RoundKeys& rk, cudaStream_t st);

// One graph work unit of a batched launch: one state plane of one job.
struct GraphUnit {
  uint64_t* n;
  uint64_t* p;
  const int32_t* nbr;
  const int32_t* bu;
  const int32_t* bv;
  const uint32_t* bid;
  int z;
  uint32_t word0;  // global index of the plane's first word
  uint32_t t_base, t_end;
  RoundKeys rk;
};
// Class cls of sweep t_base + sweep_offset for every unit (all share V and m).
cudaError_t launch_graph_class_batch(const GraphUnit* units_dev, const int64_t* prefix_dev,
                                     const int64_t* first_dev, int nunits, int64_t total_edges,
                                     int V, int m, uint32_t cls, uint32_t sweep_offset,
                                     cudaStream_t s);

struct InitScratch {
  uint32_t* hist;      // [R][256]
  uint64_t* pre_key;   // [R] decided high bits of the threshold key
  uint32_t* pre_idx;   // [R] decided high bits of the threshold site
  int64_t* krem;       // [R] rank still to place inside the current bucket
  int32_t* unresolved; // [1] any replica whose threshold key is tied
  // optional: room for per-replica candidate lists (the staging plane, idle
  // during init); null or too small -> every pass scans all sites
  uint32_t* cand;
  size_t cand_bytes;
};
cudaError_t launch_init(const Planes& pl, const InitScratch& s, int R, int64_t K,
                        const RoundKeys& rk, cudaStream_t st);

// canonical [W][N] <-> device [P][N][V] (sites in the plane order of xs)
cudaError_t launch_to_device(const uint64_t* canonical, uint64_t* device_layout, int64_t N, int P,
                             int V, int xs, const int32_t* inv, cudaStream_t st);
cudaError_t launch_to_canonical(const uint64_t* device_layout, uint64_t* canonical, int64_t N,
                                int P, int V, int xs, const int32_t* inv, cudaStream_t st);

// Group kernels of three-dimensional lattices (ka_cubic_stream.cu): one-word
// planes in split-row order, d = 3, L % 4 == 0, L <= 128.
bool stream_supported(int d, int L);
// whether a context of P one-word planes runs them (else the general kernel)
bool stream_preferred(int d, int L, int P);
// planes one launch of these kernels takes
int stream_planes_per_launch(int L, int P);
// Group (mu, par) of sweep t on planes q0 .. q0 + nq - 1.
cudaError_t launch_stream_group(const Planes& pl, int q0, int nq, int L, int m, int mu, int par,
                                uint32_t t, const RoundKeys& rk, cudaStream_t st);
// Batched group launches: one table entry (stream_unit_bytes() bytes, filled
// on the host by stream_unit_fill) per plane of every job of one side L and
// activation number m; entries whose sweep t_base + sweep_offset reaches
// t_end idle.
size_t stream_unit_bytes();
void stream_unit_fill(void* unit, uint64_t* n, uint64_t* p, uint32_t word0, uint32_t t_base,
                      uint32_t t_end, const RoundKeys& rk);
cudaError_t launch_stream_batch(const void* units_dev, int nunits, int L, int m, int mu, int par,
                                uint32_t sweep_offset, cudaStream_t st);

cudaError_t launch_observe(const Planes& pl, int R, unsigned long long* counts_dev,
                           cudaStream_t st);

}  // namespace ka
