// ka_topology.cu -- host construction of lattices, random regular graphs and
// their bond classes.  Runs once per context, before any kernel.
//
//  * Periodic cubic lattice (used by the edge-gather path; the pencil kernel
//    needs no tables): class c = (2 mu + p) * 4 + a holds the bonds
//    (x, x + e_mu) with x_mu = a mod 4 and the other coordinates summing to
//    p mod 2, bond id = base site.
//  * Random z-regular graph (section 2.1, Bollobas' configuration model):
//    shuffle the N z stubs with Fisher-Yates (Lemire's bounded integers on
//    Philox words, counter (attempt, 0xFFFFFFFE, k, draw) keyed by the graph
//    seed), pair stubs (2q, 2q+1), and reject the whole attempt on a
//    self-loop or repeated edge.  Pairs are final as soon as the shuffle has
//    passed them, so a bad attempt is abandoned early; the accepted graph is
//    the same either way.  Attempts run on several host threads; the graph
//    kept is always that of the lowest-numbered simple attempt.
//  * Layered random graph (section 5.2): M copies of the periodic cubic
//    lattice; for every base bond (i, i + e_mu) the M links between the
//    copies of i and of j = i + e_mu are rewired by a uniform permutation of
//    the copies (Fisher-Yates from the top; step k draws a uniform integer in
//    [0, k] by Lemire's method on counter (i, 0xFFFFFFFD, mu << 16 | k,
//    draw)), independently per bond.  Vertex a N + i is site i of copy a.
//  * Bond classes of a graph: greedy strong edge colouring of the edges
//    (u < v, lexicographic ids) in id order; classes in ascending colour.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <thread>

#include "ka_internal.cuh"

namespace ka {
namespace {

struct StubRng {
  RoundKeys rk;
  uint32_t attempt;
  // uniform integer in [0, range) for shuffle step k
  uint64_t below(uint32_t k, uint64_t range) const {
    uint32_t draw = 0;
    uint64_t x = lo64(philox(make_uint4(attempt, kTagGraph, k, draw), rk));
    unsigned __int128 prod = (unsigned __int128)x * range;
    uint64_t low = (uint64_t)prod;
    if (low < range) {
      const uint64_t floor = (0 - range) % range;
      while (low < floor) {
        ++draw;
        x = lo64(philox(make_uint4(attempt, kTagGraph, k, draw), rk));
        prod = (unsigned __int128)x * range;
        low = (uint64_t)prod;
      }
    }
    return (uint64_t)(prod >> 64);
  }
};

// Edge ids and classes of a simple z-regular graph with sorted rows.
std::string colour_graph(Topology& t) {
  const int64_t N = t.N;
  const int z = t.z;
  const int64_t E = N * z / 2;
  // first edge id of every vertex u: edges (u, v > u) in row order
  std::vector<int64_t> first(N + 1, 0);
  for (int64_t u = 0; u < N; ++u) {
    int up = 0;
    for (int s = 0; s < z; ++s) up += t.nbr[u * z + s] > u;
    first[u + 1] = first[u] + up;
  }
  if (first[N] != E) return "graph edge count mismatch";
  std::vector<int32_t> eu(E), ev(E);
  // incident edge ids per (vertex, slot)
  std::vector<int64_t> inc((size_t)N * z);
  for (int64_t u = 0; u < N; ++u) {
    int64_t id = first[u];
    for (int s = 0; s < z; ++s) {
      const int32_t v = t.nbr[u * z + s];
      if (v > u) {
        eu[id] = (int32_t)u;
        ev[id] = v;
        inc[u * z + s] = id++;
      }
    }
  }
  for (int64_t u = 0; u < N; ++u)
    for (int s = 0; s < z; ++s) {
      const int32_t v = t.nbr[u * z + s];
      if (v < u) {
        // id of (v, u): position of u among v's upper neighbours
        int64_t id = first[v];
        for (int r = 0; r < z; ++r) {
          const int32_t w = t.nbr[(int64_t)v * z + r];
          if (w == u) break;
          if (w > v) ++id;
        }
        inc[u * z + s] = id;
      }
    }
  std::vector<int32_t> col(E, -1);
  int32_t ncol = 0;
  std::vector<int64_t> stamp(64 * 8 + 8, -1);  // colour -> last edge that used it
  for (int64_t e = 0; e < E; ++e) {
    const int64_t ends[2] = {eu[e], ev[e]};
    auto mark = [&](int64_t w) {
      for (int s = 0; s < z; ++s) {
        const int64_t f = inc[w * z + s];
        if (f < e) stamp[col[f]] = e;
      }
    };
    for (int k = 0; k < 2; ++k) {
      mark(ends[k]);
      for (int s = 0; s < z; ++s) mark(t.nbr[ends[k] * z + s]);
    }
    int32_t c = 0;
    while (stamp[c] == e) ++c;
    col[e] = c;
    ncol = std::max(ncol, c + 1);
  }
  // counting sort by colour, stable in edge id
  t.class_off.assign(ncol + 1, 0);
  for (int64_t e = 0; e < E; ++e) t.class_off[col[e] + 1]++;
  for (int32_t c = 0; c < ncol; ++c) t.class_off[c + 1] += t.class_off[c];
  std::vector<int64_t> pos(t.class_off.begin(), t.class_off.end() - 1);
  t.bu.resize(E);
  t.bv.resize(E);
  t.bid.resize(E);
  for (int64_t e = 0; e < E; ++e) {
    const int64_t k = pos[col[e]]++;
    t.bu[k] = eu[e];
    t.bv[k] = ev[e];
    t.bid[k] = e;
  }
  return "";
}

}  // namespace

std::string build_cubic_tables(int d, int L, Topology& t) {
  if (d < 1 || d > 4 || L < 4 || L % 4) return "cubic lattice needs 1 <= d <= 4, L >= 4, L % 4 == 0";
  int64_t stride[5] = {1, 1, 1, 1, 1};
  for (int k = 1; k <= d; ++k) stride[k] = stride[k - 1] * L;
  const int64_t N = stride[d];
  const int z = 2 * d;
  t.N = N;
  t.z = z;
  t.nbr.resize((size_t)N * z);
  for (int64_t i = 0; i < N; ++i)
    for (int k = 0; k < d; ++k) {
      const int64_t x = (i / stride[k]) % L;
      const int64_t up = (x == L - 1) ? i - (L - 1) * stride[k] : i + stride[k];
      const int64_t dn = (x == 0) ? i + (L - 1) * stride[k] : i - stride[k];
      t.nbr[i * z + 2 * k] = (int32_t)up;
      t.nbr[i * z + 2 * k + 1] = (int32_t)dn;
    }
  const int nclass = (d == 1) ? 4 : 8 * d;
  t.class_off.assign(nclass + 1, 0);
  t.bu.clear();
  t.bv.clear();
  t.bid.clear();
  for (int c = 0; c < nclass; ++c) {
    const int mu = c / 8, par = (c / 4) & 1, a = c & 3;
    t.class_off[c] = (int64_t)t.bu.size();
    for (int64_t i = 0; i < N; ++i) {
      int64_t rest = i, perp = 0, xmu = 0;
      for (int k = 0; k < d; ++k) {
        const int64_t x = rest % L;
        rest /= L;
        if (k == mu)
          xmu = x;
        else
          perp += x;
      }
      if ((xmu & 3) != a || (perp & 1) != par) continue;
      t.bu.push_back((int32_t)i);
      t.bv.push_back(t.nbr[i * z + 2 * mu]);
      t.bid.push_back(i);
    }
  }
  t.class_off[nclass] = (int64_t)t.bu.size();
  return "";
}

namespace {

// One attempt of the configuration model.  Returns true, with the rows of
// the graph in adj, when the pairing is simple.  An attempt gives up early
// once a lower-numbered attempt has succeeded (`best`), since it can no
// longer be the one that is kept.
bool rrg_attempt(int64_t N, int z, const RoundKeys& rk, uint32_t att,
                 const std::atomic<int64_t>& best, std::vector<uint32_t>& stub,
                 std::vector<int32_t>& adj, std::vector<uint8_t>& deg) {
  const int64_t M = N * z;
  StubRng rng;
  rng.rk = rk;
  rng.attempt = att;
  for (int64_t s = 0; s < M; ++s) stub[s] = (uint32_t)s;
  std::fill(deg.begin(), deg.end(), 0);
  for (int64_t k = M - 1; k >= 1; --k) {
    if ((k & 0xFFFF) == 0 && best.load(std::memory_order_relaxed) < (int64_t)att) return false;
    const int64_t j = (int64_t)rng.below((uint32_t)k, (uint64_t)(k + 1));
    std::swap(stub[k], stub[j]);
    // the pair (k, k+1) for even k, and the pair (0, 1) after step 1, is final
    int64_t q0;
    if ((k & 1) == 0)
      q0 = k;
    else if (k == 1)
      q0 = 0;
    else
      continue;
    const int64_t a = stub[q0] / z, b = stub[q0 + 1] / z;
    if (a == b) return false;
    for (int s = 0; s < deg[a]; ++s)
      if (adj[a * z + s] == b) return false;
    adj[a * z + deg[a]++] = (int32_t)b;
    adj[b * z + deg[b]++] = (int32_t)a;
  }
  return true;
}

}  // namespace

// The attempts are independent (each has its own counter range), so they run
// on several host threads; the graph kept is that of the lowest-numbered
// successful attempt, exactly as in a serial loop over attempts.
std::string build_rrg(int64_t N, int z, uint64_t graph_seed, Topology& t) {
  if (N < 2 || z < 1 || z > 8 || z >= N || (N * z) % 2 || N * z > 0xFFFFFFFFLL)
    return "random regular graph needs N >= 2, 1 <= z <= 8, z < N, N z even, N z < 2^32";
  const int64_t M = N * z;
  const RoundKeys rk = round_keys(graph_seed);
  const int64_t max_attempts = 1 << 22;
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int nthreads = (int)std::min<int64_t>(std::min<unsigned>(hw, 16u), std::max<int64_t>(1, M >> 15));
  std::atomic<int64_t> next{0}, best{max_attempts};
  std::vector<int32_t> result;
  std::mutex mu;
  auto worker = [&]() {
    std::vector<uint32_t> stub(M);
    std::vector<int32_t> adj((size_t)N * z);
    std::vector<uint8_t> deg(N);
    for (;;) {
      const int64_t att = next.fetch_add(1);
      if (att >= best.load()) return;
      if (!rrg_attempt(N, z, rk, (uint32_t)att, best, stub, adj, deg)) continue;
      std::lock_guard<std::mutex> lock(mu);
      if (att < best.load()) {
        best.store(att);
        result.swap(adj);
        adj.assign((size_t)N * z, 0);
      }
      return;
    }
  };
  if (nthreads == 1) {
    worker();
  } else {
    std::vector<std::thread> pool;
    for (int i = 0; i < nthreads; ++i) pool.emplace_back(worker);
    for (auto& th : pool) th.join();
  }
  if (best.load() >= max_attempts) return "random regular graph: no simple graph within the attempt limit";
  for (int64_t v = 0; v < N; ++v) std::sort(result.begin() + v * z, result.begin() + (v + 1) * z);
  t.N = N;
  t.z = z;
  t.nbr.swap(result);
  t.attempts = (int)std::min<int64_t>(best.load() + 1, 0x7FFFFFFF);
  return colour_graph(t);
}

std::string build_graph(int64_t N, int z, const int32_t* nbr, Topology& t) {
  if (!nbr) return "KA_GRAPH needs a neighbour list";
  if (N < 2 || z < 1 || z > 8 || z >= N || N * z > 0xFFFFFFFFLL)
    return "graph needs N >= 2, 1 <= z <= 8, z < N";
  t.N = N;
  t.z = z;
  t.nbr.assign(nbr, nbr + (size_t)N * z);
  for (int64_t v = 0; v < N; ++v) {
    auto row = t.nbr.begin() + v * z;
    std::sort(row, row + z);
    for (int s = 0; s < z; ++s) {
      const int32_t w = row[s];
      if (w < 0 || w >= N) return "graph: neighbour index out of range";
      if (w == v) return "graph: self-loop";
      if (s > 0 && row[s - 1] == w) return "graph: repeated edge";
    }
  }
  // symmetry: w in row v  <=>  v in row w
  for (int64_t v = 0; v < N; ++v)
    for (int s = 0; s < z; ++s) {
      const int32_t w = t.nbr[v * z + s];
      const auto row = t.nbr.begin() + (int64_t)w * z;
      if (!std::binary_search(row, row + z, (int32_t)v)) return "graph: neighbour list not symmetric";
    }
  return colour_graph(t);
}

}  // namespace ka

namespace ka {

std::string build_layered(int d, int L, int M, uint64_t graph_seed, int32_t* nbr) {
  if (d < 1 || d > 4 || L < 3 || M < 1 || M >= 65536)
    return "layered graph needs 1 <= d <= 4, L >= 3, 1 <= M < 65536";
  int64_t N = 1;
  for (int k = 0; k < d; ++k) N *= L;
  const int z = 2 * d;
  if ((int64_t)M * N * z > 0x7FFFFFFFLL) return "layered graph: M L^d 2d must stay below 2^31";
  const RoundKeys rk = round_keys(graph_seed);
  // uniform integer in [0, range) from the words of counter (c0, tag, c2, draw)
  auto bounded = [&rk](uint32_t c0, uint32_t c2, uint64_t range) -> uint64_t {
    uint32_t draw = 0;
    uint64_t x = lo64(philox(make_uint4(c0, kTagLayer, c2, draw), rk));
    unsigned __int128 prod = (unsigned __int128)x * range;
    uint64_t low = (uint64_t)prod;
    if (low < range) {
      const uint64_t floor = (0 - range) % range;
      while (low < floor) {
        ++draw;
        x = lo64(philox(make_uint4(c0, kTagLayer, c2, draw), rk));
        prod = (unsigned __int128)x * range;
        low = (uint64_t)prod;
      }
    }
    return (uint64_t)(prod >> 64);
  };
  // bonds are independent and each writes its own slots (the up slot along
  // mu of the copies of i, the down slot of the copies of j): split the
  // base sites over threads
  auto work = [&](int64_t i0, int64_t i1) {
    std::vector<int32_t> perm(M);
    for (int64_t i = i0; i < i1; ++i) {
      int64_t stride = 1;
      for (int mu = 0; mu < d; ++mu, stride *= L) {
        const int64_t x = (i / stride) % L;
        const int64_t j = (x == L - 1) ? i - (int64_t)(L - 1) * stride : i + stride;
        for (int a = 0; a < M; ++a) perm[a] = a;
        for (int k = M - 1; k >= 1; --k) {
          const int r = (int)bounded((uint32_t)i, ((uint32_t)mu << 16) | (uint32_t)k,
                                     (uint64_t)(k + 1));
          std::swap(perm[k], perm[r]);
        }
        for (int a = 0; a < M; ++a) {
          const int64_t u = (int64_t)a * N + i, v = (int64_t)perm[a] * N + j;
          nbr[u * z + 2 * mu] = (int32_t)v;
          nbr[v * z + 2 * mu + 1] = (int32_t)u;
        }
      }
    }
  };
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int64_t nt = std::min<int64_t>(std::min<unsigned>(hw, 16u),
                                       std::max<int64_t>(1, N * M / 65536));
  if (nt <= 1) {
    work(0, N);
  } else {
    std::vector<std::thread> pool;
    for (int64_t t = 0; t < nt; ++t) pool.emplace_back(work, N * t / nt, N * (t + 1) / nt);
    for (auto& th : pool) th.join();
  }
  return "";
}

}  // namespace ka

extern "C" ka_status ka_layered_graph(int32_t d, int32_t L, int32_t M, uint64_t graph_seed,
                                      int32_t* nbr) {
  if (!nbr) return KA_EINVAL;
  return ka::build_layered(d, L, M, graph_seed, nbr).empty() ? KA_OK : KA_EINVAL;
}

namespace ka {

void bfs_order(int64_t N, int z, const int32_t* nbr, std::vector<int32_t>& perm,
               std::vector<int32_t>& inv) {
  perm.assign((size_t)N, -1);
  inv.assign((size_t)N, 0);
  int64_t head = 0, tail = 0;  // inv doubles as the queue
  for (int64_t root = 0; root < N; ++root) {
    if (perm[root] >= 0) continue;
    perm[root] = (int32_t)tail;
    inv[tail++] = (int32_t)root;
    while (head < tail) {
      const int32_t x = inv[head++];
      for (int k = 0; k < z; ++k) {
        const int32_t y = nbr[(int64_t)x * z + k];
        if (perm[y] < 0) {
          perm[y] = (int32_t)tail;
          inv[tail++] = y;
        }
      }
    }
  }
}

void relabel_tables(const Topology& t, int z, const std::vector<int32_t>& perm,
                    std::vector<int32_t>& nbr, std::vector<int32_t>& bu, std::vector<int32_t>& bv,
                    std::vector<uint32_t>& bid) {
  const int64_t N = (int64_t)perm.size();
  nbr.resize(t.nbr.size());
  for (int64_t x = 0; x < N; ++x)
    for (int k = 0; k < z; ++k)
      nbr[(int64_t)perm[x] * z + k] = perm[t.nbr[(int64_t)x * z + k]];
  const size_t E = t.bu.size();
  bu.resize(E);
  bv.resize(E);
  bid.resize(E);
  std::vector<std::pair<int32_t, int64_t>> key;
  for (int64_t c = 0; c + 1 < (int64_t)t.class_off.size(); ++c) {
    const int64_t a = t.class_off[c], b = t.class_off[c + 1];
    key.clear();
    for (int64_t e = a; e < b; ++e)
      key.emplace_back(std::min(perm[t.bu[e]], perm[t.bv[e]]), e);
    std::sort(key.begin(), key.end());
    for (int64_t k = 0; k < b - a; ++k) {
      const int64_t e = key[k].second;
      bu[a + k] = perm[t.bu[e]];
      bv[a + k] = perm[t.bv[e]];
      bid[a + k] = (uint32_t)t.bid[e];
    }
  }
}

}  // namespace ka
