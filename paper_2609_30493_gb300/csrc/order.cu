// Coherent harvest schedule.  The paper finds that the beams of neighbouring
// points share few evaluations but many targets: in a block of points that
// form a subtree of SAT tree 0, most targets are evaluated by eight or more
// of its queries (Section 5.5, Table 6), so a kernel that serves one load of
// a target to all of them removes most of the memory traffic (the
// column-batched loads the paper bounds near 2x).  On the GPU the searches
// in flight at one time share the L2 cache, so claiming the searches of a
// block in the preorder of tree 0 makes the co-scheduled queries neighbours
// and lets one read of a target row from HBM serve several of them.
//
// The rows of a block are independent given S_b (Section 4), so the order in
// which its searches run changes nothing but the traffic: the graph is the
// same for every schedule.
//
// Preorder: depths by pointer jumping, nodes bucketed by depth, subtree sizes
// summed bottom-up one depth per launch, preorder positions handed out
// top-down one depth per launch (siblings in the order their atomic adds
// land, so the preorder is valid but not unique).  Then the preorder sequence
// is split into the blocks p mod B, stably, with one count and one scatter
// pass over tiles of 1024 positions.
#include <algorithm>
#include <vector>

#include "internal.h"

namespace fg {
namespace {

constexpr int kThreads = 256;
constexpr int kTile = 1024;
constexpr int kMaxBlocks = 64;
constexpr int kMaxRounds = 32;

int grid_of(int64_t m) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((m + kThreads - 1) / kThreads, (int64_t)device_sms() * 32));
}

__global__ void jump_init_kernel(int64_t n, const int32_t* parent, int32_t* anc, int32_t* dep) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t u = parent[i];
    if (u < 0 || u >= n) u = -1;
    anc[i] = u;
    dep[i] = u >= 0 ? 1 : 0;
  }
}

// One round of pointer jumping: dep[v] is the number of edges from v up to
// anc[v] (-1 once v's root is passed).  st[0] |= some ancestor is left,
// st[1] = max over rounds of the depths (saturated at 2^30, which only a
// parent array with a cycle reaches).
__global__ void jump_step_kernel(int64_t n, const int32_t* anc_in, const int32_t* dep_in,
                                 int32_t* anc_out, int32_t* dep_out, uint32_t* st) {
  bool live = false;
  uint32_t dmax = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    if (i < n) {
      const int32_t a = anc_in[i];
      int32_t an = -1;
      int64_t dn = dep_in[i];
      if (a >= 0) {
        an = anc_in[a];
        dn += dep_in[a];
        if (dn > (1ll << 30)) dn = 1ll << 30;
      }
      anc_out[i] = an;
      dep_out[i] = (int32_t)dn;
      live |= an >= 0;
      dmax = max(dmax, (uint32_t)dn);
    }
  }
  live = __any_sync(0xffffffffu, live);
  for (int o = 16; o; o >>= 1) dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  if ((threadIdx.x & 31) == 0) {
    if (live) atomicOr(st, 1u);
    atomicMax(st + 1, dmax);
  }
}

// Adds one to cnt[key] for every valid lane, one atomic per distinct key of
// the warp; returns the lane's rank among the lanes of its key and, in
// *base, the count before the warp's add (only when want_base).
__device__ __forceinline__ uint32_t warp_count(int32_t key, bool valid, uint32_t* cnt,
                                               bool want_base, uint32_t* base) {
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(0xffffffffu, valid ? key : -1);
  const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
  uint32_t b = 0;
  if (valid && rank == 0) b = atomicAdd(&cnt[key], (uint32_t)__popc(peers));
  if (want_base) b = __shfl_sync(0xffffffffu, b, __ffs(peers) - 1);
  *base = b;
  return rank;
}

__global__ void level_count_kernel(int64_t n, const int32_t* dep, uint32_t* cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    uint32_t unused;
    warp_count(i < n ? dep[i] : 0, i < n, cnt, false, &unused);
  }
}

__global__ void level_scatter_kernel(int64_t n, const int32_t* dep, const int64_t* loff,
                                     uint32_t* cur, int32_t* lvl) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    const int32_t L = i < n ? dep[i] : 0;
    uint32_t b;
    const uint32_t r = warp_count(L, i < n, cur, true, &b);
    if (i < n) lvl[loff[L] + b + r] = (int32_t)i;
  }
}

__global__ void fill_one_kernel(int64_t n, uint32_t* v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = 1u;
}

// Subtree sizes: the nodes of one depth add their sizes into their parents.
__global__ void subtree_up_kernel(const int32_t* lvl, int64_t beg, int64_t m,
                                  const int32_t* parent, uint32_t* size) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = lvl[beg + k];
    atomicAdd(&size[parent[v]], size[v]);
  }
}

// Preorder positions of the nodes of one depth: a node takes the next free
// range of its parent's subtree (the range starts after the parent itself).
// Roots (depth 0) take ranges of a global cursor.
__global__ void preorder_down_kernel(const int32_t* lvl, int64_t beg, int64_t m,
                                     const int32_t* parent, const uint32_t* size,
                                     uint32_t* cur, uint32_t* root_cur, int32_t* pre) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = lvl[beg + k];
    const int32_t u = root_cur ? -1 : parent[v];
    if (u < 0)
      pre[v] = (int32_t)atomicAdd(root_cur, size[v]);
    else
      pre[v] = pre[u] + 1 + (int32_t)atomicAdd(&cur[u], size[v]);
  }
}

__global__ void invert_kernel(int64_t n, const int32_t* pre, int32_t* seq) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    seq[pre[i]] = (int32_t)i;
}

// Points of each block per tile of the preorder sequence, block-major.
__global__ void __launch_bounds__(kTile) block_count_kernel(int64_t n, const int32_t* seq, int nb,
                                                            int64_t ntiles, uint32_t* tcnt) {
  __shared__ uint32_t c[kMaxBlocks];
  if (threadIdx.x < kMaxBlocks) c[threadIdx.x] = 0;
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)kTile + threadIdx.x;
  if (i < n) atomicAdd(&c[seq[i] % nb], 1u);
  __syncthreads();
  if (threadIdx.x < nb) tcnt[(int64_t)threadIdx.x * ntiles + blockIdx.x] = c[threadIdx.x];
}

// Stable split of the preorder sequence into the blocks: a point's place is
// its tile's offset for its block plus the points of its block before it in
// the tile.  qorder holds query indices i of point b + i * nb.
__global__ void __launch_bounds__(kTile) block_scatter_kernel(int64_t n, const int32_t* seq,
                                                              int nb, int64_t ntiles,
                                                              const int64_t* toff,
                                                              int32_t* qorder) {
  __shared__ uint32_t wc[kTile / 32][kMaxBlocks];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < (kTile / 32) * kMaxBlocks; k += kTile) (&wc[0][0])[k] = 0;
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)kTile + threadIdx.x;
  const int32_t v = i < n ? seq[i] : -1;
  const int bk = v >= 0 ? v % nb : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, bk);
  const uint32_t r = __popc(peers & ((1u << lane) - 1u));
  if (bk >= 0 && r == 0) wc[w][bk] = __popc(peers);
  __syncthreads();
  if (bk >= 0) {
    uint32_t before = r;
    for (int w2 = 0; w2 < w; ++w2) before += wc[w2][bk];
    qorder[toff[(int64_t)bk * ntiles + blockIdx.x] + before] = (v - bk) / nb;
  }
}

template <typename T>
cudaError_t alloc_async(T** p, int64_t count, cudaStream_t s) {
  return cudaMallocAsync(reinterpret_cast<void**>(p), sizeof(T) * std::max<int64_t>(count, 1), s);
}

}  // namespace

int g_coherent = 2;  // 0: id order, 1: tree-0 preorder, 2: preorder when X exceeds the L2 cache

int coherent_schedule(int64_t n, const int32_t* parent, int nb, int max_depth, int32_t* pre,
                      int32_t* qorder, cudaStream_t s, bool* ok) {
  *ok = false;
  if (nb < 1 || nb > kMaxBlocks || n < 1) return 0;
  int32_t *anc[2] = {nullptr, nullptr}, *dep[2] = {nullptr, nullptr}, *lvl = nullptr;
  uint32_t *size = nullptr, *cur = nullptr, *st = nullptr, *cnt = nullptr, *tcnt = nullptr;
  int64_t *loff = nullptr, *toff = nullptr, *tmp = nullptr;
  auto release = [&]() {
    void* ps[] = {anc[0], anc[1], dep[0], dep[1], lvl, size, cur, st, cnt, tcnt, loff, toff, tmp};
    for (void* q : ps)
      if (q) cudaFreeAsync(q, s);
  };
#define ORD_CUDA(call)                                                          \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      release();                                                                \
      return cuda_fail(e_, #call " at " __FILE__ ":" FG_STR(__LINE__));         \
    }                                                                           \
  } while (0)
  ORD_CUDA(alloc_async(&anc[0], n, s));
  ORD_CUDA(alloc_async(&anc[1], n, s));
  ORD_CUDA(alloc_async(&dep[0], n, s));
  ORD_CUDA(alloc_async(&dep[1], n, s));
  ORD_CUDA(alloc_async(&st, 3, s));
  ORD_CUDA(cudaMemsetAsync(st, 0, 3 * sizeof(uint32_t), s));
  jump_init_kernel<<<grid_of(n), kThreads, 0, s>>>(n, parent, anc[0], dep[0]);
  note_launch();
  // depths: rounds in batches of four between host checks
  int round = 0;
  uint32_t hst[2] = {1u, 0u};
  while (hst[0] && round < kMaxRounds) {
    for (int k = 0; k < 4 && round < kMaxRounds; ++k, ++round) {
      ORD_CUDA(cudaMemsetAsync(st, 0, sizeof(uint32_t), s));
      jump_step_kernel<<<grid_of(n), kThreads, 0, s>>>(n, anc[round & 1], dep[round & 1],
                                                       anc[(round + 1) & 1],
                                                       dep[(round + 1) & 1], st);
      note_launch();
    }
    ORD_CUDA(cudaGetLastError());
    ORD_CUDA(cudaMemcpyAsync(hst, st, sizeof(hst), cudaMemcpyDeviceToHost, s));
    ORD_CUDA(cudaStreamSynchronize(s));
  }
  const int32_t* depth = dep[round & 1];
  const int64_t D = hst[1];
  if (hst[0] || D > max_depth) {  // not a tree, or too deep for one launch per depth
    release();
    return 0;
  }
  // nodes bucketed by depth
  ORD_CUDA(alloc_async(&cnt, D + 1, s));
  ORD_CUDA(alloc_async(&loff, D + 2, s));
  ORD_CUDA(alloc_async(&lvl, n, s));
  const int64_t ntiles = (n + kTile - 1) / kTile;
  ORD_CUDA(alloc_async(&tmp, scan_tmp_elems(std::max<int64_t>(D + 1, nb * ntiles)), s));
  ORD_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (D + 1), s));
  level_count_kernel<<<grid_of(n), kThreads, 0, s>>>(n, depth, cnt);
  note_launch();
  int rc = scan_u32(cnt, loff, D + 1, tmp, s);
  if (rc) {
    release();
    return rc;
  }
  ORD_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (D + 1), s));
  level_scatter_kernel<<<grid_of(n), kThreads, 0, s>>>(n, depth, loff, cnt, lvl);
  note_launch();
  std::vector<int64_t> hoff(D + 2);
  ORD_CUDA(cudaMemcpyAsync(hoff.data(), loff, sizeof(int64_t) * (D + 2), cudaMemcpyDeviceToHost,
                           s));
  // subtree sizes, deepest level first
  ORD_CUDA(alloc_async(&size, n, s));
  ORD_CUDA(alloc_async(&cur, n, s));
  fill_one_kernel<<<grid_of(n), kThreads, 0, s>>>(n, size);
  note_launch();
  ORD_CUDA(cudaMemsetAsync(cur, 0, sizeof(uint32_t) * n, s));
  ORD_CUDA(cudaStreamSynchronize(s));
  for (int64_t L = D; L >= 1; --L) {
    const int64_t m = hoff[L + 1] - hoff[L];
    if (!m) continue;
    subtree_up_kernel<<<grid_of(m), kThreads, 0, s>>>(lvl, hoff[L], m, parent, size);
    note_launch();
  }
  // preorder positions, roots first
  for (int64_t L = 0; L <= D; ++L) {
    const int64_t m = hoff[L + 1] - hoff[L];
    if (!m) continue;
    preorder_down_kernel<<<grid_of(m), kThreads, 0, s>>>(lvl, hoff[L], m, parent, size, cur,
                                                         L == 0 ? st + 2 : nullptr, pre);
    note_launch();
  }
  ORD_CUDA(cudaGetLastError());
  // the preorder sequence, split into the blocks
  int32_t* seq = anc[0];
  invert_kernel<<<grid_of(n), kThreads, 0, s>>>(n, pre, seq);
  note_launch();
  ORD_CUDA(alloc_async(&tcnt, nb * ntiles, s));
  ORD_CUDA(alloc_async(&toff, nb * ntiles + 1, s));
  block_count_kernel<<<(unsigned)ntiles, kTile, 0, s>>>(n, seq, nb, ntiles, tcnt);
  note_launch();
  rc = scan_u32(tcnt, toff, nb * ntiles, tmp, s);
  if (rc) {
    release();
    return rc;
  }
  block_scatter_kernel<<<(unsigned)ntiles, kTile, 0, s>>>(n, seq, nb, ntiles, toff, qorder);
  note_launch();
  ORD_CUDA(cudaGetLastError());
  release();
#undef ORD_CUDA
  *ok = true;
  return 0;
}

}  // namespace fg
