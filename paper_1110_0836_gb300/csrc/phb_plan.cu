// Plan set-up, workspace layout, status helpers and the device-wide scan.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "phb_internal.cuh"

namespace phb {

namespace {
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
}  // namespace

int64_t scan_blocks(int64_t count) { return (count + kScanTile - 1) / kScanTile; }

Grid make_grid(const phb_plan* p) {
  Grid g;
  for (int a = 0; a < 3; ++a) {
    g.lo[a] = p->box.lo[a];
    g.len[a] = p->box.len[a];
    g.inv_cell[a] = 1.0 / p->cell[a];
    g.inv_ncell[a] = 1.0 / p->ncell[a];
    g.cell[a] = p->cell[a];
    g.periodic[a] = p->box.periodic[a] ? 1 : 0;
    g.lenf[a] = static_cast<float>(p->box.len[a]);
    g.inv_lenf[a] = p->box.periodic[a] ? static_cast<float>(1.0 / p->box.len[a]) : 0.f;
    g.ncell[a] = p->ncell[a];
    g.nbrick[a] = p->nbrick[a];
  }
  g.hbits = p->hilbert_bits;
  g.tile = p->tile;
  g.stage_cap = p->stage_cap;
  g.schedule = p->schedule;
  g.ell = p->ell_width;
  g.n = static_cast<int32_t>(p->n);
  g.rf_factor = p->rf_factor;
  g.skin = p->skin;
  g.lambda_min = p->lambda_min;
  g.lambda_max = p->lambda_max;
  g.screen_margin = static_cast<float>(p->screen_margin);
  g.capacity = p->nbr_capacity;
  return g;
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 148;
  }
  return sms;
}

size_t l2_bytes() {
  static int l2 = 0;
  if (!l2) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess || l2 <= 0)
      l2 = 64 << 20;
  }
  return static_cast<size_t>(l2);
}

phb_status launch_status(cudaError_t e) {
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? PHB_OK : PHB_ERR_CUDA;
}

phb_status check_common(const phb_plan* plan, const void* ws, size_t ws_bytes, size_t need) {
  if (!plan || plan->n <= 0 || plan->ws_bytes == 0) return PHB_ERR_INVALID_ARG;
  if (!ws) return PHB_ERR_INVALID_ARG;
  if (ws_bytes < need) return PHB_ERR_WORKSPACE;
  return PHB_OK;
}

// ------------------------------------------------------------------ scan
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Exclusive block scan of one value per thread; returns the block total.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* smem_warp, T& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) smem_warp[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T w = lane < nw ? smem_warp[lane] : T(0);
    T wi = warp_incl_scan(w);
    if (lane < nw) smem_warp[lane] = wi - w;
    if (lane == 31) smem_warp[32] = wi;
  }
  __syncthreads();
  T res = inc - v + smem_warp[wid];
  total = smem_warp[32];
  __syncthreads();
  return res;
}

template <typename TIn, typename TOut>
__global__ void __launch_bounds__(kScanThreads) k_scan_tile(const TIn* in, TOut* out, int64_t count,
                                                            int64_t* bsum) {
  __shared__ int64_t sw[33];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t run = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    v[k] = i < count ? static_cast<int64_t>(in[i]) : 0;
    run += v[k];
  }
  int64_t total;
  int64_t pre = block_excl_scan<int64_t>(run, sw, total);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    if (i < count) out[i] = static_cast<TOut>(pre);
    pre += v[k];
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_sums(int64_t* bsum, int64_t nb) {
  __shared__ int64_t sw[33];
  int64_t carry = 0;
  for (int64_t c0 = 0; c0 < nb; c0 += blockDim.x) {
    int64_t i = c0 + threadIdx.x;
    int64_t v = i < nb ? bsum[i] : 0;
    int64_t total;
    int64_t pre = block_excl_scan<int64_t>(v, sw, total);
    if (i < nb) bsum[i] = pre + carry;
    carry += total;
  }
}

template <typename TOut>
__global__ void k_scan_add(TOut* out, int64_t count, const int64_t* bsum) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < count) out[i] += static_cast<TOut>(bsum[i / kScanTile]);
}

// Two-launch scan for up to kScanTwoMax tiles: the tiles' sums, then every
// tile scans itself after adding up the sums of the tiles before it (at most
// kScanTwoMax values, from L2).  Every launch is as wide as the array, which
// a one-block scan of a short array is not.  In place is fine (a tile is read
// before it is written, and only by its own block).
constexpr int64_t kScanTwoMax = 256;

template <typename TIn>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const TIn* in, int64_t count,
                                                              int64_t* bsum) {
  __shared__ int64_t sw[33];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + threadIdx.x * kScanItems;
  int64_t run = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + k;
    run += i < count ? static_cast<int64_t>(in[i]) : 0;
  }
  int64_t total;
  block_excl_scan<int64_t>(run, sw, total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

template <typename TIn, typename TOut>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const TIn* in, TOut* out, int64_t count,
                                                             const int64_t* bsum) {
  __shared__ int64_t sw[33];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t run = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + k;
    v[k] = i < count ? static_cast<int64_t>(in[i]) : 0;
    run += v[k];
  }
  // the sums of the tiles before this one (blockIdx.x <= kScanTwoMax - 1 < kScanThreads)
  int64_t before;
  {
    const int64_t b = threadIdx.x < blockIdx.x ? bsum[threadIdx.x] : 0;
    block_excl_scan<int64_t>(b, sw, before);
  }
  int64_t total;
  int64_t pre = block_excl_scan<int64_t>(run, sw, total) + before;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + k;
    if (i < count) out[i] = static_cast<TOut>(pre);
    pre += v[k];
  }
}

template <typename TIn, typename TOut>
cudaError_t scan_impl(const TIn* in, TOut* out, int64_t count, int64_t* bsum, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int64_t nb = scan_blocks(count);
  if (nb <= kScanTwoMax) {
    k_scan_reduce<TIn><<<static_cast<unsigned>(nb), kScanThreads, 0, st>>>(in, count, bsum);
    note_launch();
    k_scan_apply<TIn, TOut><<<static_cast<unsigned>(nb), kScanThreads, 0, st>>>(in, out, count, bsum);
    note_launch();
    return cudaGetLastError();
  }
  k_scan_tile<TIn, TOut><<<static_cast<unsigned>(nb), kScanThreads, 0, st>>>(in, out, count, bsum);
  note_launch();
  k_scan_sums<<<1, 1024, 0, st>>>(bsum, nb);
  note_launch();
  k_scan_add<TOut><<<static_cast<unsigned>((count + 255) / 256), 256, 0, st>>>(out, count, bsum);
  note_launch();
  return cudaGetLastError();
}

cudaError_t scan_exclusive_i32_to_i64(const int32_t* in, int64_t* out, int64_t count,
                                      int64_t* block_sums, cudaStream_t st) {
  return scan_impl<int32_t, int64_t>(in, out, count, block_sums, st);
}

cudaError_t scan_exclusive_i32(int32_t* data, int64_t count, int64_t* block_sums, cudaStream_t st) {
  return scan_impl<int32_t, int32_t>(data, data, count, block_sums, st);
}

}  // namespace phb

using namespace phb;

extern "C" phb_status phb_plan_init(phb_plan* p) {
  if (!p) return PHB_ERR_INVALID_ARG;
  p->ws_bytes = 0;
  if (p->n <= 0 || p->n >= (int64_t(1) << 31) - 1) return PHB_ERR_INVALID_ARG;
  if (!(p->rf_factor > 0) || !(p->skin >= 0) || !(p->lambda_min > 0) ||
      !(p->lambda_max >= p->lambda_min) || !std::isfinite(p->lambda_max))
    return PHB_ERR_INVALID_ARG;
  if (p->nbr_capacity < 0) return PHB_ERR_INVALID_ARG;
  double xmax = 0, lmax = 0;
  for (int a = 0; a < 3; ++a) {
    if (!(p->box.len[a] > 0) || !std::isfinite(p->box.len[a]) || !std::isfinite(p->box.lo[a]))
      return PHB_ERR_INVALID_ARG;
    xmax = std::max(xmax, std::max(std::fabs(p->box.lo[a]), std::fabs(p->box.lo[a] + p->box.len[a])));
    lmax = std::max(lmax, p->box.len[a]);
  }
  const double rmin = p->rf_factor * p->lambda_min + p->skin;
  const double rmax = p->rf_factor * p->lambda_max + p->skin;
  for (int a = 0; a < 3; ++a)
    if (p->box.periodic[a] && !(rmax < 0.5 * p->box.len[a])) return PHB_ERR_INVALID_ARG;
  double frac = p->cell_frac > 0 ? p->cell_frac : 1.0;
  double h = frac * rmin;
  // at most 1023 cells per axis (10-bit packed coordinates), 2^26 cells in all
  for (int a = 0; a < 3; ++a) h = std::max(h, p->box.len[a] / 1023.0);
  for (int it = 0; it < 64; ++it) {
    double cells = 1;
    for (int a = 0; a < 3; ++a) cells *= std::max(1.0, std::floor(p->box.len[a] / h));
    if (cells <= double(1 << 26)) break;
    h *= 1.1;
  }
  int maxb = 1;
  for (int a = 0; a < 3; ++a) {
    int nc = static_cast<int>(std::max(1.0, std::floor(p->box.len[a] / h)));
    nc = std::min(nc, 1023);
    p->ncell[a] = nc;
    p->cell[a] = p->box.len[a] / nc;
    p->nbrick[a] = (nc + 3) / 4;
    maxb = std::max(maxb, p->nbrick[a]);
  }
  int hb = 0;
  while ((1 << hb) < maxb) ++hb;
  p->hilbert_bits = hb;
  const int64_t nkeys = (int64_t(1) << (3 * hb)) * 64;
  if (nkeys >= (int64_t(1) << 31) - 2) return PHB_ERR_INVALID_ARG;
  p->nkeys = nkeys;
  if (p->tile == 0) p->tile = 128;
  if (p->tile != 64 && p->tile != 128) return PHB_ERR_INVALID_ARG;
  // default stage: the largest that keeps two 128-thread fit CTAs (254
  // registers each) per SM: 2 x (29 KB parked right-hand sides + 48 B per
  // record) within 227 KB; the 64-thread tiles run four CTAs per SM
  if (p->stage_cap == 0) p->stage_cap = p->tile == 128 ? 1750 : 768;
  if (p->stage_cap < 64 || p->stage_cap > 2048) return PHB_ERR_INVALID_ARG;
  p->ntiles = static_cast<int32_t>((p->n + p->tile - 1) / p->tile);
  if (p->schedule != 0 && p->schedule != 1) return PHB_ERR_INVALID_ARG;
  // default scratch row: ~51 neighbours at r_f = 2.3 lambda and uniform
  // density; where lambda varies, a coarse particle next to a refined region
  // gathers up to (lambda_max / lambda_min)^3 times more (275 at a 2x jump):
  // rows too short send those lists through a second search in the
  // compaction, so varying-lambda plans get 256 slots
  if (p->ell_width == 0) p->ell_width = p->lambda_max > 1.26 * p->lambda_min ? 256 : 128;
  if (p->ell_width < 8 || p->ell_width > 1024) return PHB_ERR_INVALID_ARG;
  // FP32 screen: bound of |d32 - d| per component is 2^-24 (2X + 3L); two
  // components' worth of safety on top, times sqrt(3) for the norm.
  p->screen_margin = 8.0 * std::sqrt(3.0) * std::ldexp(1.0, -24) * (2.0 * xmax + 3.0 * lmax);

  const int64_t n = p->n, cap = std::max<int64_t>(p->nbr_capacity, 1);
  size_t sz[R_COUNT] = {0};
  sz[R_MISC] = 64 * 4;
  sz[R_KEYS] = n * 4;
  sz[R_PERM] = n * 4;
  sz[R_INV] = n * 4;
  sz[R_CELL] = (nkeys + 1) * 4;
  sz[R_CURSOR] = nkeys * 4;
  sz[R_SCAN] = (scan_blocks(std::max<int64_t>(nkeys + 1, n + 1)) + 1) * 8;
  sz[R_SPOS] = 3 * n * 8;
  sz[R_SLAM] = n * 8;
  sz[R_SU] = 8 * n * 8;
  sz[R_REC] = n * kRec * 4;
  sz[R_SCREEN] = n * 16;
  sz[R_NCNT] = (n + 1) * 4;
  sz[R_OFF] = (n + 1) * 8;
  sz[R_IDX] = cap * 4;
  sz[R_LIDX] = cap * 2;
  sz[R_CELLC] = n * 4;
  sz[R_CLIN] = size_t(p->ncell[0]) * p->ncell[1] * p->ncell[2] * 8;
  sz[R_LSTART] = (size_t(p->ncell[0]) * p->ncell[1] * p->ncell[2] + 1) * 4;
  sz[R_LSCR] = size_t(n + 4) * 16;
  sz[R_TORDER] = size_t(p->ntiles) * 4;
  sz[R_ELL] = size_t(n) * p->ell_width * 4;
  sz[R_TPLAN] = size_t(p->ntiles) * 8;
  sz[R_TSLOT] = size_t(p->ntiles) * p->stage_cap * 4;
  sz[R_LSELF] = size_t(n) * 2;
  sz[R_TMAP] = size_t(p->ntiles) * p->tile;
  sz[R_ALIST] = size_t(n + 64) * 4;
  sz[R_AFLAG] = size_t(n + 1) * 4;
  sz[R_QUEUE] = (n + 64) * 4;  // also the export's n+1 counts
  sz[R_RQUEUE] = size_t(n) * 4;
  sz[R_RSTASH] = size_t(80 + kNF * 19) * n * 4;
  sz[R_DIAG] = size_t(3) * kDiagBlocks * 8;
  size_t off = 0;
  for (int r = R_MISC; r <= R_DIAG; ++r) {
    p->ws_off[r] = off;
    off += align256(sz[r]);
  }
  p->ws_off[R_END_COMMON] = off;
  // PC-step regions
  size_t pc = off;
  p->ws_off[R_PC_F0] = pc;
  pc += align256(size_t(8) * n * 8);
  p->ws_off[R_PC_F1] = pc;
  pc += align256(size_t(8) * n * 8);
  p->ws_off[R_PC_Y0] = pc;
  pc += align256(size_t(11) * n * 8);
  p->ws_off[R_PC_IO] = pc;
  pc += align256(size_t(12) * n * 8);
  p->ws_off[R_PC_DONE] = pc;
  pc += align256(size_t(n));
  // adjoint regions overlay the PC ones
  size_t ad = off;
  p->ws_off[R_ADJ_ROFF] = ad;
  ad += align256(size_t(n + 1) * 8);
  p->ws_off[R_ADJ_RSRC] = ad;
  ad += align256(size_t(cap) * 4);
  p->ws_off[R_ADJ_RCNT] = ad;
  ad += align256(size_t(n + 1) * 4);
  p->ws_off[R_ADJ_SCR] = ad;
  ad += align256(size_t(266) * n * 8);
  p->ws_off[R_ADJ_SELF] = ad;
  ad += align256(size_t(11) * n * 8);
  p->ws_off[R_END_PC] = pc;
  p->ws_off[R_END_ADJ] = ad;
  p->ws_off[R_END] = std::max(pc, ad);
  p->ws_bytes = p->ws_off[R_END];
  return PHB_OK;
}

extern "C" int phb_workspace_part(const phb_plan* p, int32_t part, size_t* begin, size_t* end) {
  if (!p || p->ws_bytes == 0 || !begin || !end) return 1;
  switch (part) {
    case PHB_PART_COMMON: *begin = 0; *end = p->ws_off[R_END_COMMON]; return 0;
    case PHB_PART_STEP: *begin = p->ws_off[R_END_COMMON]; *end = p->ws_off[R_END_PC]; return 0;
    case PHB_PART_ADJOINT: *begin = p->ws_off[R_END_COMMON]; *end = p->ws_off[R_END_ADJ]; return 0;
    default: return 1;
  }
}

extern "C" size_t phb_workspace_size(const phb_plan* p, int32_t op) {
  if (!p || p->ws_bytes == 0) return 0;
  (void)op;
  return p->ws_bytes;
}

extern "C" int phb_struct_sizes(int64_t* out, int32_t count) {
  if (!out || count < 1 || count > 3) return 1;
  const int64_t v[3] = {static_cast<int64_t>(sizeof(phb_box)), static_cast<int64_t>(sizeof(phb_params)),
                        static_cast<int64_t>(sizeof(phb_plan))};
  for (int k = 0; k < count; ++k) out[k] = v[k];
  return 0;
}

extern "C" const char* phb_status_string(int32_t s) {
  switch (s) {
    case PHB_OK: return "ok";
    case PHB_ERR_INVALID_ARG: return "invalid argument";
    case PHB_ERR_WORKSPACE: return "workspace too small";
    case PHB_ERR_CUDA: return "CUDA error";
    case PHB_ERR_CAPACITY: return "neighbour list capacity exceeded";
    case PHB_ERR_SKIN: return "predictor displacement exceeded half the skin";
    case PHB_WARN_FIT: return "singular fit (derivatives set to zero)";
    case PHB_ERR_TIMEOUT: return "bounded device wait timed out";
    case PHB_ERR_NONFINITE: return "non-finite value";
    default: return "unknown status";
  }
}

extern "C" phb_status phb_check(int32_t w) {
  if (w & PHB_FLAG_TIMEOUT) return PHB_ERR_TIMEOUT;
  if (w & PHB_FLAG_CAPACITY) return PHB_ERR_CAPACITY;
  if (w & (PHB_FLAG_LAMBDA_RANGE | PHB_FLAG_BAD_INDEX)) return PHB_ERR_INVALID_ARG;
  if (w & PHB_FLAG_SKIN) return PHB_ERR_SKIN;
  if (w & PHB_FLAG_NONFINITE) return PHB_ERR_NONFINITE;
  if (w & PHB_FLAG_FIT_SINGULAR) return PHB_WARN_FIT;
  return PHB_OK;
}
