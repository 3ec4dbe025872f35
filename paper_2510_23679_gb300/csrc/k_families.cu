// k_families.cu -- gene families as connected components of the Bidirectional
// Best Hit graph (phase (c) of the pipeline, "extract gene families from the
// Bidirectional Best Hits"; the refinement PanDelos applies afterwards is not
// specified, so a family here is a connected component).
//
// Union-find by minimum label: parent[i] <= i always.  Each round
//   hook      for every edge (u, v) whose roots differ, the larger root is
//             hooked under the smaller one (atomicMin, so parents only
//             decrease and concurrent hooks never form a cycle);
//   compress  every node jumps to its root.
// Rounds repeat until no edge hooks.  The root of a component is then its
// smallest node id, which is the family label (independent of edge order).
// Parent chains strictly decrease, so every chase ends within n steps.
#include <algorithm>
#include <string>

#include "pd.h"
#include "pd_host.cuh"
#include "pd_internal.cuh"

using namespace pdh;

namespace {

__device__ __forceinline__ int32_t root_of(const int32_t* parent, int32_t x) {
  int32_t p = parent[x];
  while (p != x) {
    x = p;
    p = parent[x];
  }
  return x;
}

__global__ void k_cc_init(int32_t* parent, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) parent[i] = (int32_t)i;
}

__global__ void k_cc_hook(const int32_t* __restrict__ ea, const int32_t* __restrict__ eb, uint64_t n_edges,
                          int32_t* parent, uint32_t n, int* changed, pdg::DevErr* err) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_edges;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const int32_t u = ea[e], v = eb[e];
    if (u < 0 || v < 0 || (uint32_t)u >= n || (uint32_t)v >= n) {
      pdg::raise_error(err, PD_ERR_ARG, e);
      continue;
    }
    const int32_t ru = root_of(parent, u), rv = root_of(parent, v);
    if (ru == rv) continue;
    const int32_t hi = max(ru, rv), lo = min(ru, rv);
    atomicMin(&parent[hi], lo);
    *changed = 1;
  }
}

__global__ void k_cc_compress(int32_t* parent, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    parent[i] = root_of(parent, (int32_t)i);
}

__global__ void k_cc_count_roots(const int32_t* __restrict__ parent, uint32_t n, unsigned int* count) {
  uint32_t mine = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    mine += parent[i] == (int32_t)i ? 1u : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31u) == 0 && mine) atomicAdd(count, mine);
}

unsigned grid_of(uint64_t items, unsigned per_block, unsigned cap) {
  uint64_t b = (items + per_block - 1) / per_block;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, cap));
}

#define PD_KLAUNCH(name, ...)           \
  do {                                  \
    CK(pdg::launch_begin(&c->L, name)); \
    __VA_ARGS__;                        \
    CK(pdg::launch_end(&c->L, name));   \
  } while (0)

// Rounds allowed before giving up.  Every round that hooks joins at least two
// trees, so n rounds always suffice; real graphs converge in a few.
constexpr int kMaxRounds = 4096;

pd_status components_impl(pd_ctx* c, const int32_t* a, const int32_t* b, uint64_t n_edges, uint32_t n_nodes,
                          int32_t* label, uint32_t* n_components) {
  if ((n_edges && (!a || !b)) || (n_nodes && !label)) return fail(c, PD_ERR_ARG, "null argument");
  if (n_nodes > 0x7FFFFFFFu) return fail(c, PD_ERR_ARG, "too many nodes");
  CK(cudaSetDevice(c->device));
  Buf parent, da, db, flag, cnt;
  ALLOC(parent, sizeof(int32_t) * std::max<uint32_t>(n_nodes, 1));
  const int32_t* ea = a;
  const int32_t* eb = b;
  if (n_edges && !is_device_ptr(a)) {
    ALLOC(da, sizeof(int32_t) * n_edges);
    CK(cudaMemcpyAsync(da.p, a, sizeof(int32_t) * n_edges, cudaMemcpyHostToDevice, c->stream));
    ea = da.as<int32_t>();
  }
  if (n_edges && !is_device_ptr(b)) {
    ALLOC(db, sizeof(int32_t) * n_edges);
    CK(cudaMemcpyAsync(db.p, b, sizeof(int32_t) * n_edges, cudaMemcpyHostToDevice, c->stream));
    eb = db.as<int32_t>();
  }
  ALLOC(flag, sizeof(int));
  ALLOC(cnt, sizeof(unsigned int));
  if (n_nodes)
    PD_KLAUNCH("cc_init", (k_cc_init<<<grid_of(n_nodes, 256, 152u * 8u), 256, 0, c->stream>>>(parent.as<int32_t>(),
                                                                                                 n_nodes)));
  int round = 0;
  for (; n_edges && n_nodes && round < kMaxRounds; ++round) {
    CK(cudaMemsetAsync(flag.p, 0, sizeof(int), c->stream));
    PD_KLAUNCH("cc_hook", (k_cc_hook<<<grid_of(n_edges, 256, 152u * 16u), 256, 0, c->stream>>>(
                              ea, eb, n_edges, parent.as<int32_t>(), n_nodes, flag.as<int>(), c->d_err)));
    PD_KLAUNCH("cc_compress", (k_cc_compress<<<grid_of(n_nodes, 256, 152u * 8u), 256, 0, c->stream>>>(
                                  parent.as<int32_t>(), n_nodes)));
    int h = 0;
    CK(cudaMemcpyAsync(&h, flag.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    pd_status st = check_dev_err(c);  // synchronizes
    if (st != PD_OK) return st;
    if (!h) break;
  }
  if (round == kMaxRounds) return fail(c, PD_ERR_INTERNAL, "connected components did not converge");
  unsigned int roots = 0;
  CK(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned int), c->stream));
  if (n_nodes)
    PD_KLAUNCH("cc_count", (k_cc_count_roots<<<grid_of(n_nodes, 256, 152u * 8u), 256, 0, c->stream>>>(
                               parent.as<int32_t>(), n_nodes, cnt.as<unsigned int>())));
  CK(cudaMemcpyAsync(&roots, cnt.p, sizeof(roots), cudaMemcpyDeviceToHost, c->stream));
  pd_status st;
  if ((st = copy_out(c, label, parent.p, sizeof(int32_t) * n_nodes)) != PD_OK) return st;
  CK(cudaStreamSynchronize(c->stream));
  if (n_components) *n_components = roots;
  return PD_OK;
}

}  // namespace

PD_API pd_status pd_components(pd_ctx* c, const int32_t* a, const int32_t* b, uint64_t n_edges, uint32_t n_nodes,
                               int32_t* label, uint32_t* n_components) {
  if (!c) return PD_ERR_ARG;
  try {
    return components_impl(c, a, b, n_edges, n_nodes, label, n_components);
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_components");
  }
}

PD_API pd_status pd_families(pd_ctx* c, const pd_bbh_set* S, uint32_t n_genes, int32_t* family,
                             uint32_t* n_families) {
  if (!c || !S) return PD_ERR_ARG;
  try {
    return components_impl(c, S->a.as<int32_t>(), S->b.as<int32_t>(), S->n, n_genes, family, n_families);
  } catch (const std::bad_alloc&) {
    return fail(c, PD_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(c, PD_ERR_INTERNAL, "exception in pd_families");
  }
}
