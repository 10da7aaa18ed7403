// sort.cu -- stable sort of one species' particles by tile key with
// compaction of removed particles, and the (species, tile, chunk) work list
// of the tiled push.
//
// Key = tile index (cells grouped in tile_r x tile_t blocks, row-major over
// tiles); removed particles get the key ntiles and sort last, and so does a
// cell index outside the grid (never produced by the push; only a caller's
// input can hold one), which is also reported through a flag word.  The sort is an
// LSD radix sort over 8-bit digits of (key, index) pairs.  Each pass: per-block
// digit histograms (kSortBlock elements per block), one exclusive scan over the
// digit-major histogram matrix, and a stable scatter in which every element's
// rank inside its block comes from warp match masks, so equal keys keep their
// order (the result equals a stable sort by key).  The particle payload moves
// once, in a final gather.
#include <algorithm>
#include <mutex>

#include "../../include/hff.h"
#include "hff_common.cuh"

namespace hff {


// the divisions by nt, tile_r and tile_t by multiplication (FastDiv): the
// first radix pass computes the key of every slot twice (histogram and
// scatter), and three run-time integer divisions cost several times the rest
__device__ __forceinline__ uint32_t tile_key(int cell, int nt, const FastDiv &dnt, const FastDiv &dtr,
                                             const FastDiv &dtt, int ntt, int64_t ncells, uint32_t dead) {
  if (cell < 0 || cell >= ncells) return dead;
  const uint32_t i = fastdiv(dnt, (uint32_t)cell), j = (uint32_t)cell - i * (uint32_t)nt;
  return fastdiv(dtr, i) * (uint32_t)ntt + fastdiv(dtt, j);
}

struct SortArgs {
  const int32_t *cell;      // first pass: keys are computed from the cells
  const uint32_t *keys_in;  // later passes
  const uint32_t *idx_in;
  uint32_t *keys_out, *idx_out;
  uint32_t *hist;
  int64_t n;
  int64_t ncells;           // nr * nt: larger cell indices are invalid input
  unsigned *bad;            // flag word: bad_bit is or-ed in for an invalid cell
  unsigned bad_bit;
  int nb, shift, nt, tile_r, tile_t, ntt;
  FastDiv dnt, dtr, dtt;    // divisions by nt, tile_r, tile_t
  uint32_t dead;
  bool first;
};

__device__ __forceinline__ uint32_t load_key(const SortArgs &a, int64_t e) {
  return a.first ? tile_key(a.cell[e], a.nt, a.dnt, a.dtr, a.dtt, a.ntt, a.ncells, a.dead) : a.keys_in[e];
}

__global__ void __launch_bounds__(kSortThreads) k_hist(SortArgs a) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortBlock;
  bool bad = false;
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t e = base + r * kSortThreads + threadIdx.x;
    if (e < a.n) {
      atomicAdd(&h[(load_key(a, e) >> a.shift) & 255u], 1u);
      if (a.first && a.cell[e] >= a.ncells) bad = true;
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(a.bad, a.bad_bit);
  __syncthreads();
  a.hist[(int64_t)threadIdx.x * a.nb + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of n words in place: block sums, scan of the sums, apply
__global__ void __launch_bounds__(1024) k_scan_sums(const uint32_t *x, int64_t n, uint32_t *part) {
  __shared__ uint32_t w[32];
  const int64_t base = (int64_t)blockIdx.x * kScanBlock;
  uint32_t s = 0;
  for (int k = threadIdx.x; k < kScanBlock; k += 1024) {
    const int64_t e = base + k;
    if (e < n) s += x[e];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t v = w[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *w, uint32_t &total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) w[wid] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t t = (threadIdx.x < nw) ? w[threadIdx.x] : 0u;
    uint32_t z = t;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
      if (threadIdx.x >= o) z += y;
    }
    w[threadIdx.x] = z - t;  // exclusive warp offsets
    if (threadIdx.x == 31) w[32] = z;
  }
  __syncthreads();
  const uint32_t r = w[wid] + x - v;
  total = w[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(1024) k_scan_parts(uint32_t *part, int m) {
  __shared__ uint32_t w[33];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int seg = 0; seg < m; seg += 1024) {
    const int k = seg + threadIdx.x;
    const uint32_t v = (k < m) ? part[k] : 0u;
    uint32_t tot;
    const uint32_t ex = block_excl_scan(v, w, tot);
    if (k < m) part[k] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024) k_scan_apply(uint32_t *x, int64_t n, const uint32_t *part) {
  __shared__ uint32_t w[33];
  __shared__ uint32_t carry;
  const int64_t base = (int64_t)blockIdx.x * kScanBlock;
  if (threadIdx.x == 0) carry = part[blockIdx.x];
  __syncthreads();
  for (int seg = 0; seg < kScanBlock; seg += 1024) {
    const int64_t e = base + seg + threadIdx.x;
    const uint32_t v = (e < n) ? x[e] : 0u;
    uint32_t tot;
    const uint32_t ex = block_excl_scan(v, w, tot);
    if (e < n) x[e] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
}

// stable scatter: element order inside a block is (round, warp, lane)
__global__ void __launch_bounds__(kSortThreads) k_scatter(SortArgs a) {
  constexpr int kW = kSortThreads / 32;
  __shared__ uint32_t s_base[256];        // global offset of each digit for this block
  __shared__ uint16_t s_cnt[kW][256];     // per-warp digit counts of the round
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  s_base[threadIdx.x] = a.hist[(int64_t)threadIdx.x * a.nb + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kSortBlock;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int r = 0; r < kSortItems; ++r) {
    for (int w = 0; w < kW; ++w) s_cnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t e = base + r * kSortThreads + threadIdx.x;
    const bool ok = e < a.n;
    uint32_t key = 0, val = 0, d = 256;
    if (ok) {
      key = load_key(a, e);
      val = a.first ? (uint32_t)e : a.idx_in[e];
      d = (key >> a.shift) & 255u;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt_mask);
    if (ok && rank == 0) s_cnt[wid][d] = (uint16_t)__popc(peers);
    __syncthreads();
    // thread t owns digit t: exclusive offsets over the warps, then advance
    {
      uint32_t acc = 0;
      for (int w = 0; w < kW; ++w) {
        const uint32_t c = s_cnt[w][threadIdx.x];
        s_cnt[w][threadIdx.x] = (uint16_t)acc;
        acc += c;
      }
      __syncthreads();
      if (ok) {
        const uint32_t pos = s_base[d] + s_cnt[wid][d] + rank;
        a.keys_out[pos] = key;
        a.idx_out[pos] = val;
      }
      __syncthreads();
      s_base[threadIdx.x] += acc;
    }
    __syncthreads();
  }
}

template <typename R>
__global__ void __launch_bounds__(256) k_gather(Species<R> src, Species<R> dst, const uint32_t *idx,
                                                const uint32_t *keys, uint32_t dead, int64_t n,
                                                long long *count, long long *count_sorted, int species) {
  // live count = first index whose key is dead (keys are sorted)
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    if (keys[q] == dead) {
      if (q == 0 || keys[q - 1] != dead) { count[species] = q; count_sorted[species] = q; }
      dst.cell[q] = -1;  // every slot past the live count holds a removed particle
      continue;
    }
    if (q == n - 1) { count[species] = n; count_sorted[species] = n; }
    const uint32_t k = idx[q];
    dst.cell[q] = src.cell[k];
    dst.xo[q] = src.xo[k]; dst.yo[q] = src.yo[k];
    dst.ur[q] = src.ur[k]; dst.ut[q] = src.ut[k]; dst.up[q] = src.up[k];
    dst.w[q] = src.w[k];
  }
}

// One pass over the sorted keys of a sort whose payload moves later: the
// live count, cell = -1 in the removed slots of the destination, and the
// tile bounds.  Four keys per thread (one 16-byte load; the keys buffer is
// 256-byte aligned), plus the neighbours of the group.
__global__ void __launch_bounds__(256) k_finish_bounds(int32_t *dst_cell, const uint32_t *keys, uint32_t dead,
                                                       int64_t n, long long *count, long long *count_sorted,
                                                       int species, int *start, int *end) {
  const int64_t groups = (n + 3) / 4;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < groups; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q0 = 4 * g;
    uint32_t k[6];  // k[0] = key before the group, k[5] = key after it
    if (q0 + 3 < n) {
      const uint4 v = *reinterpret_cast<const uint4 *>(keys + q0);
      k[1] = v.x; k[2] = v.y; k[3] = v.z; k[4] = v.w;
    } else {
      for (int e = 0; e < 4; ++e) k[1 + e] = (q0 + e < n) ? keys[q0 + e] : dead;
    }
    k[0] = q0 > 0 ? keys[q0 - 1] : dead;
    k[5] = q0 + 4 < n ? keys[q0 + 4] : dead;
    for (int e = 0; e < 4; ++e) {
      const int64_t q = q0 + e;
      if (q >= n) break;
      const uint32_t c = k[1 + e];
      if (c == dead) {
        if (q == 0 || k[e] != dead) { count[species] = q; count_sorted[species] = q; }
        dst_cell[q] = -1;
        continue;
      }
      if (q == n - 1) { count[species] = n; count_sorted[species] = n; }
      if (q == 0 || k[e] != c) start[c] = (int)q;
      if (q == n - 1 || k[2 + e] != c) end[c] = (int)(q + 1);
    }
  }
}

// the deferred payload gather: slots below the (already compacted) count
template <typename R>
__global__ void __launch_bounds__(256) k_gather_live(Species<R> src, Species<R> dst, const uint32_t *idx,
                                                     const long long *count, int species) {
  const int64_t n = count[species];
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = idx[q];
    dst.cell[q] = src.cell[k];
    dst.xo[q] = src.xo[k]; dst.yo[q] = src.yo[k];
    dst.ur[q] = src.ur[k]; dst.ut[q] = src.ut[k]; dst.up[q] = src.up[k];
    dst.w[q] = src.w[k];
  }
}

__global__ void k_set_count(long long *count, long long *count_sorted, int species, long long v) {
  count[species] = v;
  count_sorted[species] = v;
}

// tile bounds from the sorted keys: start[k] .. end[k]
__global__ void k_bounds(const uint32_t *keys, int64_t n, uint32_t dead, int *start, int *end) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = keys[q];
    if (k == dead) continue;
    if (q == 0 || keys[q - 1] != k) start[k] = (int)q;
    if (q == n - 1 || keys[q + 1] != k) end[k] = (int)(q + 1);
  }
}

// append ceil(count/chunk) items per non-empty tile of one species
__global__ void __launch_bounds__(1024) k_worklist(const int *start, const int *end, int ntiles, int species,
                                                   int chunk, int4 *items, int *n_items, int max_items,
                                                   bool first, unsigned *status) {
  __shared__ uint32_t w[33];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = first ? 0u : (uint32_t)*n_items;
  __syncthreads();
  for (int seg = 0; seg < ntiles; seg += 1024) {
    const int k = seg + threadIdx.x;
    int cnt = 0;
    if (k < ntiles) cnt = end[k] - start[k];
    const uint32_t ni = cnt > 0 ? (uint32_t)((cnt + chunk - 1) / chunk) : 0u;
    uint32_t tot;
    const uint32_t ex = block_excl_scan(ni, w, tot);
    for (uint32_t c = 0; c < ni; ++c) {
      const uint32_t slot = carry + ex + c;
      if ((int)slot < max_items) {
        const int s0 = start[k] + (int)c * chunk;
        const int len = min(chunk, end[k] - s0);
        items[slot] = make_int4(species, k, s0, len);
      } else {
        atomicOr(status, kStWorklist);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_items = (int)min((int)carry, max_items);
}

static int bits_for(uint32_t v) {
  int b = 0;
  while ((1ull << b) <= v) ++b;
  return b;
}

template <typename R>
void launch_sort_species(const Params<R> &p, int s, Species<R> dst, const SortScratch &ss, cudaStream_t st,
                         bool gather) {
  // The slot count lives on the device, so (to stay capturable in a CUDA
  // graph) the passes run over the whole capacity; every slot at or past the
  // count holds cell = -1 (kept so by hff_init, this gather and injection),
  // so those slots sort last as removed particles.
  const int64_t n = ss.cap;
  const uint32_t dead = (uint32_t)ss.ntiles;
  const int nbits = bits_for(dead);
  const int passes = (nbits + 7) / 8;
  const int nb = (int)((n + kSortBlock - 1) / kSortBlock);
  const int64_t hn = (int64_t)nb * 256;
  const int nparts = (int)((hn + kScanBlock - 1) / kScanBlock);
  SortArgs a{};
  a.cell = p.sp[s].cell;
  a.n = n;
  a.ncells = (int64_t)p.nr * p.nt;
  a.bad = p.status;
  a.bad_bit = kStBadCell;
  a.nb = nb;
  a.nt = p.nt; a.tile_r = p.tile_r; a.tile_t = p.tile_t; a.ntt = p.ntt;
  a.dnt = make_fastdiv((uint32_t)p.nt); a.dtr = make_fastdiv((uint32_t)p.tile_r); a.dtt = make_fastdiv((uint32_t)p.tile_t);
  a.dead = dead;
  a.hist = ss.hist;
  uint32_t *ko = ss.keys_a, *io = ss.idx_a, *ki = ss.keys_b, *ii = ss.idx_b;
  for (int pass = 0; pass < passes; ++pass) {
    a.first = (pass == 0);
    a.shift = 8 * pass;
    a.keys_in = ki; a.idx_in = ii;
    a.keys_out = ko;
    // the last pass leaves the sorted order in this species' own buffer
    a.idx_out = (pass == passes - 1) ? const_cast<uint32_t *>(p.sidx[s]) : io;
    k_hist<<<nb, kSortThreads, 0, st>>>(a);
    k_scan_sums<<<nparts, 1024, 0, st>>>(ss.hist, hn, ss.part);
    k_scan_parts<<<1, 1024, 0, st>>>(ss.part, nparts);
    k_scan_apply<<<nparts, 1024, 0, st>>>(ss.hist, hn, ss.part);
    k_scatter<<<nb, kSortThreads, 0, st>>>(a);
    uint32_t *t = ki; ki = ko; ko = t;
    t = ii; ii = io; io = t;
  }
  // ki holds the sorted keys, p.sidx[s] the sorted order
  k_set_count<<<1, 1, 0, st>>>(p.count, p.count_sorted, s, (long long)n);
  cudaMemsetAsync(ss.tile_start, 0, sizeof(int) * (ss.ntiles + 1), st);
  cudaMemsetAsync(ss.tile_end, 0, sizeof(int) * (ss.ntiles + 1), st);
  if (gather) {
    k_gather<R><<<1216, 256, 0, st>>>(p.sp[s], dst, p.sidx[s], ki, dead, n, p.count, p.count_sorted, s);
    k_bounds<<<1216, 256, 0, st>>>(ki, n, dead, ss.tile_start, ss.tile_end);
  } else {
    k_finish_bounds<<<1216, 256, 0, st>>>(dst.cell, ki, dead, n, p.count, p.count_sorted, s, ss.tile_start,
                                          ss.tile_end);
  }
}

// Loaded particles: a cell index at or past nr * nt is invalid input; the
// particle is removed (cell = -1) and kStBadCell latched.
__global__ void k_check_cells(int32_t *cell, int64_t n, int64_t ncells, unsigned *status) {
  bool bad = false;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    if (cell[q] >= ncells) { cell[q] = -1; bad = true; }
  if (bad) atomicOr(status, kStBadCell);
}

void launch_check_cells(int32_t *cell, int64_t n, int64_t ncells, unsigned *status, cudaStream_t st) {
  if (n > 0) k_check_cells<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(cell, n, ncells, status);
}

template <typename R>
void launch_materialize(const Params<R> &p, int s, cudaStream_t st) {
  k_gather_live<R><<<1216, 256, 0, st>>>(p.src[s], p.sp[s], p.sidx[s], p.count, s);
}

template <typename R>
void launch_worklist(const Params<R> &p, const SortScratch *ss, const WorkList &wl, int species, int first,
                     cudaStream_t st) {
  k_worklist<<<1, 1024, 0, st>>>(ss->tile_start, ss->tile_end, ss->ntiles, species, wl.chunk, wl.items,
                                 wl.n_items, wl.max_items, first != 0, p.status);
}

#define HFF_INST(R)                                                                                   \
  template void launch_sort_species<R>(const Params<R> &, int, Species<R>, const SortScratch &, cudaStream_t, bool); \
  template void launch_materialize<R>(const Params<R> &, int, cudaStream_t); \
  template void launch_worklist<R>(const Params<R> &, const SortScratch *, const WorkList &, int, int,   \
                                   cudaStream_t);
HFF_INST(float)
HFF_INST(double)
#undef HFF_INST

// ------------------------------------------------- allocation-free variant
// hff_tile_order_noalloc runs the same radix passes with its scratch in a
// fixed device array instead of memory passed in or allocated, for callers
// that may not allocate device memory at all.  The paper has no counterpart.
namespace noalloc {

constexpr int64_t kMaxN = HFF_NOALLOC_MAX_PARTICLES;
constexpr int64_t kMaxBlocks = (kMaxN + kSortBlock - 1) / kSortBlock;
constexpr int64_t kMaxHist = kMaxBlocks * 256;
constexpr int64_t kMaxParts = (kMaxHist + kScanBlock - 1) / kScanBlock;
// keys_a | keys_b | idx_a | idx_b | histogram | block sums | live count,
// invalid-cell flag
constexpr int64_t kWords = 4 * kMaxN + kMaxHist + kMaxParts + 64;

// One copy per device, alive until the process exits; shared by every call.
static __device__ __align__(256) uint32_t g_scratch[kWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t *g_addr[kMaxDevices] = {};

// live count and invalid-cell flag: written afresh at the start of every call
__global__ void k_live_init(uint32_t *live, uint32_t n) {
  live[0] = n;
  live[1] = 0u;
}

// first slot holding a removed particle (keys are sorted, removed ones last)
__global__ void k_live_count(const uint32_t *keys, int64_t n, uint32_t dead, uint32_t *live) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    if (keys[q] == dead && (q == 0 || keys[q - 1] != dead)) *live = (uint32_t)q;
}

}  // namespace noalloc
}  // namespace hff

thread_local const char *hff_noalloc_err = "";

extern "C" const char *hff_noalloc_last_error(void) { return hff_noalloc_err; }

extern "C" int hff_tile_order_noalloc(const int32_t *cell, int64_t n, int32_t nr, int32_t nt, int32_t tile_r,
                                      int32_t tile_t, uint32_t *order, int64_t *n_live, void *stream) {
  using namespace hff;
  using namespace hff::noalloc;
  // an error left by earlier, unrelated work would otherwise be reported
  // (and cleared) by the check after this call's launches
  (void)cudaGetLastError();
  if (n < 0 || nr < 1 || nt < 1 || tile_r < 1 || tile_t < 1 || !n_live || (n > 0 && (!cell || !order))) {
    hff_noalloc_err = "hff_tile_order_noalloc: invalid argument";
    return HFF_ERR_ARG;
  }
  if (n > kMaxN) {
    hff_noalloc_err = "hff_tile_order_noalloc: n exceeds HFF_NOALLOC_MAX_PARTICLES";
    return HFF_ERR_CAPACITY;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    hff_noalloc_err = "hff_tile_order_noalloc: no usable current device";
    return HFF_ERR_CUDA;
  }
  uint32_t *base = nullptr;
  {
    // first call on this device: resolve the device address of the array
    // (host code only sees a stand-in symbol; the device address differs)
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void *ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) {
        hff_noalloc_err = "hff_tile_order_noalloc: cudaGetSymbolAddress failed";
        return HFF_ERR_CUDA;
      }
      g_addr[dev] = static_cast<uint32_t *>(ptr);
    }
    base = g_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int ntt = (nt + tile_t - 1) / tile_t;
  const int64_t ntiles = (int64_t)((nr + tile_r - 1) / tile_r) * ntt;
  if (ntiles >= 0x7fffffffLL) {
    hff_noalloc_err = "hff_tile_order_noalloc: too many tiles";
    return HFF_ERR_ARG;
  }
  uint32_t *keys_a = base, *keys_b = base + kMaxN, *idx_a = base + 2 * kMaxN, *idx_b = base + 3 * kMaxN;
  uint32_t *hist = base + 4 * kMaxN, *part = hist + kMaxHist, *live = part + kMaxParts;
  const uint32_t dead = (uint32_t)ntiles;
  if (n == 0) {
    *n_live = 0;
    hff_noalloc_err = "";
    return HFF_OK;
  }
  const int nbits = bits_for(dead), passes = (nbits + 7) / 8;
  const int nb = (int)((n + kSortBlock - 1) / kSortBlock);
  const int64_t hn = (int64_t)nb * 256;
  const int nparts = (int)((hn + kScanBlock - 1) / kScanBlock);
  SortArgs a{};
  a.cell = cell;
  a.n = n;
  a.ncells = (int64_t)nr * nt;
  a.bad = live + 1;
  a.bad_bit = 1u;
  a.nb = nb;
  a.nt = nt; a.tile_r = tile_r; a.tile_t = tile_t; a.ntt = ntt;
  a.dnt = make_fastdiv((uint32_t)nt); a.dtr = make_fastdiv((uint32_t)tile_r); a.dtt = make_fastdiv((uint32_t)tile_t);
  a.dead = dead;
  a.hist = hist;
  k_live_init<<<1, 1, 0, st>>>(live, (uint32_t)n);
  uint32_t *ko = keys_a, *io = idx_a, *ki = keys_b, *ii = idx_b;
  for (int pass = 0; pass < passes; ++pass) {
    a.first = (pass == 0);
    a.shift = 8 * pass;
    a.keys_in = ki; a.idx_in = ii;
    a.keys_out = ko; a.idx_out = io;
    k_hist<<<nb, kSortThreads, 0, st>>>(a);
    k_scan_sums<<<nparts, 1024, 0, st>>>(hist, hn, part);
    k_scan_parts<<<1, 1024, 0, st>>>(part, nparts);
    k_scan_apply<<<nparts, 1024, 0, st>>>(hist, hn, part);
    k_scatter<<<nb, kSortThreads, 0, st>>>(a);
    uint32_t *t = ki; ki = ko; ko = t;
    t = ii; ii = io; io = t;
  }
  // the live count and the flag were written at the start of this call
  // (previous contents of the shared array are never read)
  k_live_count<<<(int)((n + 255) / 256), 256, 0, st>>>(ki, n, dead, live);
  uint32_t h_live[2] = {0u, 0u};
  if (cudaMemcpyAsync(order, ii, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(h_live, live, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    hff_noalloc_err = "hff_tile_order_noalloc: a CUDA call failed";
    return HFF_ERR_CUDA;
  }
  if (h_live[1]) {
    hff_noalloc_err = "hff_tile_order_noalloc: a cell index is at or past nr * nt (ordered as removed)";
    return HFF_ERR_ARG;
  }
  *n_live = (int64_t)h_live[0];
  hff_noalloc_err = "";
  return HFF_OK;
}
