// Internal declarations shared by the CUDA translation units of libphurbas.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/phurbas.h"

namespace phb {

constexpr int kNF = 8;      // fields rho, Vx, Vy, Vz, Bx, By, Bz, sigma
constexpr int kRec = 24;    // floats per FP32 particle record (6 x float4)
constexpr int kDiagBlocks = 1024;  // fixed grid of the diagnostic reductions (deterministic sums)

// Workspace regions (byte offsets in plan->ws_off).  The PC-step and adjoint
// regions share storage (never used at the same time).
enum Region {
  R_MISC = 0,    // int32 [64]: 0 = FP64 route-queue length, 1 = tiles that fell back to
                 //   global gathers in the last neighbour build, 2 = same in the last
                 //   fused fit, 3 = (unused), 4 = active-subset
                 //   length, 5 = tiles refined by the last FP32-mixed fit, 6 = fits
                 //   queued for its corrected step
  R_KEYS,        // int32 [n]   cell key of each caller particle
  R_PERM,        // int32 [n]   slot -> caller index
  R_INV,         // int32 [n]   caller index -> slot
  R_CELL,        // int32 [nkeys+1] cell start (exclusive scan of counts)
  R_CURSOR,      // int32 [nkeys]   scatter cursors
  R_SCAN,        // int64 [scan blocks] block sums
  R_SPOS,        // double [3][n] positions, slot order
  R_SLAM,        // double [n]    lambda, slot order
  R_SU,          // double [8][n] fields, slot order
  R_REC,         // float [n][24] FP32 hi/lo records
  R_SCREEN,      // float4 [n]   wrapped FP32 positions for the neighbour screen
  R_NCNT,        // int32 [n+1]  neighbour counts
  R_OFF,         // int64 [n+1]  CSR offsets (slot order)
  R_IDX,         // int32 [capacity] neighbour slots
  R_LIDX,        // uint16 [capacity] neighbour index inside the tile's staged neighbourhood
  R_CELLC,       // int32 [n] packed cell coordinates of each slot (10 bits per axis)
  R_CLIN,        // int2 [cells] (first slot, count) per linear cell index (x-major)
  R_LSTART,      // int32 [cells+1] first record of each cell in linear cell order
  R_LSCR,        // float4 [n+4] screen records in linear cell order, slot in w (+ padding)
  R_TORDER,      // int32 [ntiles] tiles in descending cost class (schedule 1)
  R_ELL,         // int32 [n][ell_width] first list entries of each slot (single-pass search)
  R_TPLAN,       // int2 [ntiles] (staged particles, 1 = not staged) of each tile's neighbourhood
  R_TSLOT,       // int32 [ntiles][stage_cap] slot of every staged index of each tile
  R_LSELF,       // uint16 [n] each slot's own staged index within its tile
  R_TMAP,        // uint8 [ntiles][tile] fit thread -> tile particle, longest list first
  R_ALIST,       // int32 [n+64] slots of an active subset (ascending)
  R_AFLAG,       // int32 [n+1]  active-subset marks / their exclusive scan
  R_QUEUE,       // int32 [n]    slots routed to FP64
  R_RQUEUE,      // int32 [n]    slots of refined tiles' fits, queued for the corrected step
  R_RSTASH,      // float [80 + 8*19][n] per queued fit (queue order): its moments in the
                 //   packed pair layout, then the 19 first-solve coefficients of each field
  R_DIAG,        // double [3][kDiagBlocks] block partial sums of the mode-amplitude diagnostic
  R_PC_F0,       // double [8][n] F(Y^n) (slot order)        -- PC step
  R_PC_F1,       // double [8][n] F(Y^p) (slot order)        -- PC step
  R_PC_Y0,       // double [11][n] saved x^n, U^n (slot order) -- PC step
  R_PC_IO,       // double [12][n] pos, lambda, U (caller order) of phb_pc_step_host -- PC step
  R_PC_DONE,     // uint8 [n] slots whose U^{n+1} the corrector's fit wrote to the host -- PC step
  R_ADJ_ROFF,    // int64 [n+1] reverse-list offsets                     -- adjoint
  R_ADJ_RSRC,    // int32 [capacity] reverse lists: the particles naming each particle -- adjoint
  R_ADJ_RCNT,    // int32 [n+1] reverse-list counts / cursors            -- adjoint
  R_ADJ_SCR,     // double [n][266] per particle: seeds bbar, coefficients c then mbar -- adjoint
  R_ADJ_SELF,    // double [11][n] each particle's own adjoint terms      -- adjoint
  R_END_COMMON,  // end of the common part (prefix for RHS / derivs)
  R_END,         // end of everything
  R_END_PC,      // end of the PC-step regions
  R_END_ADJ,     // end of the adjoint regions
  R_COUNT
};
static_assert(R_COUNT <= 48, "ws_off has 48 entries");

template <typename T>
__host__ __device__ inline T* region(const phb_plan* p, void* ws, Region r) {
  return reinterpret_cast<T*>(static_cast<char*>(ws) + p->ws_off[r]);
}
template <typename T>
__host__ __device__ inline const T* region(const phb_plan* p, const void* ws, Region r) {
  return reinterpret_cast<const T*>(static_cast<const char*>(ws) + p->ws_off[r]);
}

// Plain-old-data view of the plan handed to kernels by value.
struct Grid {
  double lo[3], len[3], inv_cell[3], cell[3], inv_ncell[3];
  float lenf[3], inv_lenf[3];  // FP32 box lengths and (periodic axes) their reciprocals, else 0
  int32_t periodic[3], ncell[3], nbrick[3];
  int32_t hbits;      // Hilbert order of the brick curve
  int32_t tile;       // particles per tile
  int32_t stage_cap;  // staged records per tile
  int32_t schedule;   // 0: tiles in cell order, 1: tiles in descending cost
  int32_t ell;        // list entries kept per slot by the single-pass search
  int32_t n;
  double rf_factor, skin;
  double lambda_min, lambda_max;
  float screen_margin;
  int64_t capacity;
};

Grid make_grid(const phb_plan* p);

__device__ __forceinline__ float phb_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double phb_rsqrt(double x) { return 1.0 / sqrt(x); }

__device__ __forceinline__ void raise_flag(int32_t* status_word, int32_t bits) {
  if (status_word) atomicOr(status_word, bits);
}

// FP64 finiteness from the exponent bits, on the integer pipe.  GB300's FP64
// rate is about 1/64 of its FP32 rate, so the bookkeeping kernels keep FP64
// instructions to the arithmetic that needs them.
__device__ __forceinline__ bool finite64(double x) {
  return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000;
}

// Cell coordinate on one axis and the matching wrap count k: with
// u = floor((x - lo) / cell) (reciprocal cell edge), a periodic axis gives
// c = u - k nc, k = floor(u / nc), and the wrapped position x - k len lies in
// cell c up to the rounding of that subtraction - the cell and the wrapped
// position never disagree by a box length, also for a particle at lo + len
// exactly.  An open axis clamps c into [0, ncell) with k = 0.  The scaled
// position is formed in FP64; for |u| < 2^30 the floor, the wrap and the clamp
// are integer operations (k_zero: no wrap), further out the same steps run in
// exact integer-valued FP64.  x must be finite.
static __device__ __noinline__ int cell_wrap_fp64(const Grid& g, int a, double t, double& k_out,
                                                 bool& k_zero);

__device__ __forceinline__ int cell_wrap(const Grid& g, int a, double x, double& k_out,
                                         bool& k_zero) {
  const double t = (x - g.lo[a]) * g.inv_cell[a];
  const int nc = g.ncell[a];
  if (((__double2hiint(t) >> 20) & 0x7ff) < 1023 + 30) {
    const int u = __double2int_rd(t);
    if (g.periodic[a]) {
      if (static_cast<unsigned>(u) < static_cast<unsigned>(nc)) {
        k_zero = true;
        k_out = 0.0;
        return u;
      }
      const int k = u >= 0 ? u / nc : -((-1 - u) / nc) - 1;
      k_zero = false;
      k_out = static_cast<double>(k);
      return u - k * nc;
    }
    k_zero = true;
    k_out = 0.0;
    return u < 0 ? 0 : (u >= nc ? nc - 1 : u);
  }
  return cell_wrap_fp64(g, a, t, k_out, k_zero);
}

// cell_wrap far outside the box, out of line (not run predicated for every
// position).
static __device__ __noinline__ int cell_wrap_fp64(const Grid& g, int a, double t, double& k_out,
                                                 bool& k_zero) {
  const int nc = g.ncell[a];
  const double u = floor(t);
  if (g.periodic[a]) {
    double k = floor(u * g.inv_ncell[a]);
    double c = u - k * nc;
    if (c < 0) {
      c += nc;
      k -= 1;
    } else if (c >= nc) {
      c -= nc;
      k += 1;
    }
    k_out = k;
    k_zero = false;
    return static_cast<int>(c);
  }
  k_out = 0.0;
  k_zero = true;
  return u < 0 ? 0 : (u >= nc ? nc - 1 : static_cast<int>(u));
}

__device__ __forceinline__ int cell_coord(const Grid& g, int a, double x) {
  double k;
  bool kz;
  return cell_wrap(g, a, x, k, kz);
}

// lambda_min <= l <= lambda_max for lambda_min >= 0, on the integer pipe: the
// bit patterns of non-negative doubles order like their values; negative
// values and NaNs fall outside.
__device__ __forceinline__ bool lambda_in_range(const Grid& g, double l) {
  const long long b = __double_as_longlong(l);
  return b >= __double_as_longlong(g.lambda_min) && b <= __double_as_longlong(g.lambda_max);
}

// FP32 wrapped position x - k len from cell_wrap's outputs (the wrapped case
// out of line).
static __device__ __noinline__ float wrapped32_shift(const Grid& g, int a, double x, double k) {
  return static_cast<float>(__dsub_rn(x, __dmul_rn(k, g.len[a])));
}

__device__ __forceinline__ float wrapped32(const Grid& g, int a, double x, double k, bool k_zero) {
  if (k_zero) return __double2float_rn(x);
  return wrapped32_shift(g, a, x, k);
}

// Index of brick (x, y, z) along a 3-D Hilbert curve of order b (2^b bricks per
// axis): Skilling's transform of the axes to the transposed Hilbert integer
// (J. Skilling, AIP Conf. Proc. 707, 381 (2004)), then bit interleaving.
// Consecutive indices are face-adjacent bricks.
__host__ __device__ inline uint32_t hilbert3(uint32_t x, uint32_t y, uint32_t z, int b) {
  if (b <= 0) return 0;
  uint32_t X[3] = {x, y, z};
  const uint32_t M = 1u << (b - 1);
  for (uint32_t Q = M; Q > 1; Q >>= 1) {
    const uint32_t P = Q - 1;
    for (int i = 0; i < 3; ++i) {
      if (X[i] & Q) {
        X[0] ^= P;
      } else {
        const uint32_t t = (X[0] ^ X[i]) & P;
        X[0] ^= t;
        X[i] ^= t;
      }
    }
  }
  X[1] ^= X[0];
  X[2] ^= X[1];
  uint32_t t = 0;
  for (uint32_t Q = M; Q > 1; Q >>= 1)
    if (X[2] & Q) t ^= Q - 1;
  X[0] ^= t;
  X[1] ^= t;
  X[2] ^= t;
  uint32_t h = 0;
  for (int j = b - 1; j >= 0; --j)
    for (int i = 0; i < 3; ++i) h = (h << 1) | ((X[i] >> j) & 1u);
  return h;
}

// Cell key: 4x4x4-cell bricks ordered along the Hilbert curve, Morton order of
// the 64 cells inside a brick.  Cells that are close in space get close keys,
// so a run of consecutive particles covers a compact region.
__device__ __forceinline__ int32_t cell_key(const Grid& g, int cx, int cy, int cz) {
  const uint32_t hb = hilbert3(static_cast<uint32_t>(cx >> 2), static_cast<uint32_t>(cy >> 2),
                               static_cast<uint32_t>(cz >> 2), g.hbits);
  int x = cx & 3, y = cy & 3, z = cz & 3;
  int m = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2) | ((x & 2) << 2) | ((y & 2) << 3) | ((z & 2) << 4);
  return static_cast<int32_t>(hb * 64u + static_cast<uint32_t>(m));
}

__host__ __device__ inline int32_t pack_cell(int cx, int cy, int cz) { return cx | (cy << 10) | (cz << 20); }
__host__ __device__ inline void unpack_cell(int32_t p, int& cx, int& cy, int& cz) {
  cx = p & 1023;
  cy = (p >> 10) & 1023;
  cz = (p >> 20) & 1023;
}

// Minimum-image FP64 offset, d - len * nearbyint(d / len), correctly rounded
// at every step and without contraction (bit-identical to the definition).
// Below a quarter box length the rounded quotient is 0 and d is returned as
// it is, without the (slow) FP64 division.
__device__ __forceinline__ double min_image64(double d, double len, int periodic) {
  if (periodic && !(fabs(d) < 0.25 * len)) d = __dsub_rn(d, __dmul_rn(len, rint(__ddiv_rn(d, len))));
  return d;
}

// Squared FP64 distance ((dx*dx + dy*dy) + dz*dz), same evaluation order.
__device__ __forceinline__ double dist2_exact(const Grid& g, const double* spos, int n, int s,
                                              int t) {
  double dx = min_image64(__dsub_rn(spos[t], spos[s]), g.len[0], g.periodic[0]);
  double dy = min_image64(__dsub_rn(spos[n + t], spos[n + s]), g.len[1], g.periodic[1]);
  double dz = min_image64(__dsub_rn(spos[2 * n + t], spos[2 * n + s]), g.len[2], g.periodic[2]);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// List radius r = rf_factor * lambda + skin (two roundings, no contraction).
__device__ __forceinline__ double list_radius(const Grid& g, double lam) {
  return __dadd_rn(__dmul_rn(g.rf_factor, lam), g.skin);
}

// a - b with minimum image for FP32 hi/lo pairs (a = ah + al, b = bh + bl).
// The hi difference is split exactly (TwoSum) so that a wrap by k box
// lengths, exact by Sterbenz, loses nothing; accurate to ~1 ulp of the result.
__device__ __forceinline__ float mi_diff32(float ah, float al, float bh, float bl, float len_h,
                                           float len_l, float inv_len) {
  float s = ah - bh;
  float bp = s - ah;
  float e = (ah - (s - bp)) + (-bh - bp);
  float k = rintf(s * inv_len);
  float t = fmaf(-k, len_h, s);
  return t + (((al - bl) + e) - k * len_l);
}

// ------------------------------------------------------------ host helpers
cudaError_t scan_exclusive_i32_to_i64(const int32_t* in, int64_t* out, int64_t count,
                                      int64_t* block_sums, cudaStream_t st);
cudaError_t scan_exclusive_i32(int32_t* data, int64_t count, int64_t* block_sums, cudaStream_t st);
int64_t scan_blocks(int64_t count);

phb_status check_common(const phb_plan* plan, const void* ws, size_t ws_bytes, size_t need);
phb_status launch_status(cudaError_t e);

// Gather caller-order pos, lambda, U into slot order (FP64 copies and FP32
// hi/lo records).  U may be NULL (positions only).  y0, if not NULL, gets a
// second slot-order copy of (x, U) ([11][n]; the predictor-corrector's Y^n).
cudaError_t gather_sorted(const phb_plan* plan, const Grid& g, const double* pos,
                          const double* lambda, const double* U, void* ws, int32_t* status_word,
                          cudaStream_t st, double* y0 = nullptr);

cudaError_t build_neighbors_impl(const phb_plan* p, const double* pos, const double* lam, void* ws,
                                 int32_t* status_word, cudaStream_t st);

// FP32 hi/lo split of an FP64 value: h = v rounded to FP32, l = (v - h)
// rounded to FP32 (v - h is exact in FP64).  For 2^-74 <= |v| < 2^127 both
// come from the two 32-bit words of v with integer and FP32 operations only:
// h rounds the 53-bit significand to 24 bits (to nearest, ties to even); the
// signed remainder r (|r| <= 2^28, in units of v's last significand bit) is
// rounded once by one FMA of its exact high and low 14-bit parts and scaled
// by a power of two.  The results equal the FP64 form's, which serves zero
// and every other value.
__device__ __forceinline__ float exact_small_float(unsigned int m) {
  // m < 2^23 as an FP32 value, exactly: 2^23 + m has m in its significand
  return __uint_as_float(0x4b000000u | m) - 8388608.f;
}

// The FP64 form, out of line: inlined, the compiler would run it predicated
// for every value.
static __device__ __noinline__ void split_hl_fp64(double v, float& h, float& l) {
  h = __double2float_rn(v);
  l = __double2float_rn(v - static_cast<double>(h));
}

__device__ __forceinline__ void split_hl(double v, float& h, float& l) {
  const unsigned int hw = static_cast<unsigned int>(__double2hiint(v));
  const unsigned int lw = static_cast<unsigned int>(__double2loint(v));
  const int e = static_cast<int>((hw >> 20) & 0x7ffu);
  if (e >= 949 && e < 1150) {
    unsigned int q = 0x800000u | ((hw & 0xfffffu) << 3) | (lw >> 29);  // leading 24 bits
    const unsigned int r = lw & 0x1fffffffu;                           // the other 29
    const bool up = r > 0x10000000u || (r == 0x10000000u && (q & 1u));
    const unsigned int mag = up ? 0x20000000u - r : r;  // |remainder| <= 2^28
    q += up ? 1u : 0u;
    int eh = e - 1023;
    if (q == 0x1000000u) {
      q >>= 1;
      eh += 1;
    }
    const unsigned int sign = hw & 0x80000000u;
    h = __uint_as_float(sign | (static_cast<unsigned int>(eh + 127) << 23) | (q & 0x7fffffu));
    // the remainder's sign is the value's when rounded down, the opposite when rounded up
    const float rm = fmaf(exact_small_float(mag >> 14), 16384.f, exact_small_float(mag & 0x3fffu));
    const float lm = rm * __uint_as_float(static_cast<unsigned int>(e - 948) << 23);
    const bool neg = (sign != 0u) != up;
    l = mag == 0u ? 0.f : (neg ? -lm : lm);
    return;
  }
  split_hl_fp64(v, h, l);
}

// Write the 6-float4 record of slot s: (xh,yh,zh,0) (xl,yl,zl,0)
// (rho,sigma,Vx,Vy)_h (rho,sigma,Vx,Vy)_l (Vz,Bx,By,Bz)_h (Vz,Bx,By,Bz)_l.
__device__ __forceinline__ void write_record(float* rec, int64_t s, const double (&x)[3],
                                             const double (&u)[8]) {
  float xh[3], xl[3], uh[8], ul[8];
  for (int a = 0; a < 3; ++a) split_hl(x[a], xh[a], xl[a]);
  for (int f = 0; f < 8; ++f) split_hl(u[f], uh[f], ul[f]);
  float4* r = reinterpret_cast<float4*>(rec) + 6 * s;
  r[0] = make_float4(xh[0], xh[1], xh[2], 0.f);
  r[1] = make_float4(xl[0], xl[1], xl[2], 0.f);
  r[2] = make_float4(uh[0], uh[7], uh[1], uh[2]);
  r[3] = make_float4(ul[0], ul[7], ul[1], ul[2]);
  r[4] = make_float4(uh[3], uh[4], uh[5], uh[6]);
  r[5] = make_float4(ul[3], ul[4], ul[5], ul[6]);
}

// Fit + RHS / derivatives in slot order; outputs scattered to caller order
// through `perm` when out_perm is non-null, else written in slot order.
enum class FitMode { kRHS = 0, kDerivs = 1 };
struct FitArgs {
  Grid g;
  int32_t n;
  const int32_t* perm_in;      // slot -> caller index for zeta / eta (null: identity)
  const int32_t* perm_out;     // slot -> caller index for outputs (null: slot order)
  const double* spos;          // [3][n]
  const double* slam;          // [n]
  const double* sU;            // [8][n]
  const float* rec;            // [n][24]
  const int64_t* off;          // [n+1]
  const int32_t* idx;          // [capacity]
  double gamma;
  int32_t weight_kind;
  float cond_threshold;
  const double* zeta;          // caller order (indexed through perm_in) or null
  const double* eta;
  double c_zeta_l, c_zeta_a, c_eta;  // coefficient laws (phb_params), 0 = off
  double* dudt;                // [8][n]
  double* grad;                // [8][3][n]
  double* hess;                // [8][6][n] or null
  int32_t* fit_status;         // [n] or null
  int32_t* queue;              // FP64 route queue
  int32_t* queue_len;
  int32_t* status_word;
  // FP32-mixed corrected semi-normal-equations step: -1 off, 0 tiles whose
  // largest conditioning estimate exceeds refine_kappa, 1 every tile
  int32_t refine_mode;
  float refine_kappa;
  // the corrected step of refined tiles in k_fit_refine over a queue (sets
  // whose FP32 records fit in L2 and whose lambda varies) or inside the tile
  // (larger sets: the tile's neighbourhood is still in L2 right after its
  // main passes)
  bool refine_queued;
  int32_t* rqueue;             // [n] fits queued for the corrected step
  int32_t* rq_len;             // their count (zeroed before the launch)
  float* rstash;               // [kNM + 8*19][n] moments and first solves, queue order
  int32_t* refined_tiles;      // count of refined tiles (zeroed before the launch)
  // host-buffer step, corrector evaluation (u_host null: off): each tile
  // writes U^{n+1} = Y^n + h (F(Y^n) + F(Y^p)) of its final fits straight to
  // the caller's page-locked U_out, where a warp's slots map to nearby caller
  // indices, and marks those slots in pc_done
  double* u_host;              // mapped host [8][n], caller order
  const double* pc_y0;         // [11][n] slot order: x^n, U^n
  const double* pc_f0;         // [8][n] slot order: F(Y^n)
  const int32_t* pc_perm;      // slot -> caller index
  const uint8_t* pc_frozen;    // caller order, or null
  uint8_t* pc_done;            // [n] slot order
  double pc_h;                 // dt / 2
};

// What the corrector's fit of the host-buffer step needs for its direct
// write of U^{n+1} (FitArgs.u_host and the pc_ fields).
struct HostU {
  double* u_host;
  const double* y0;
  const double* f0;
  const int32_t* perm;
  const uint8_t* frozen;
  uint8_t* done;
  double h;
};

// Fused FP32-mixed fit over all slots (list == null, staged tiles) or over
// the slots list[0 .. *list_len) (at most list_cap; unstaged path).
cudaError_t launch_fit_mixed(const FitArgs& a, FitMode mode, const int2* tplan, const int32_t* tslot,
                             const uint16_t* lself, const uint8_t* tmap, const uint16_t* lidx,
                             int32_t* fallback_count, const int32_t* order,
                             const int32_t* list, const int32_t* list_len, int64_t list_cap,
                             cudaStream_t st);
// Tensor-core experiment: Gram matrices on mma.sync (3xTF32) into gram
// [214][n], then the solve and right-hand side (tile 128 only).
cudaError_t launch_fit_tc(const FitArgs& a, const int2* tplan, const int32_t* tslot,
                          const uint16_t* lself, const uint8_t* tmap, const uint16_t* lidx,
                          float* gram, cudaStream_t st);
// Fit arguments of a plan, parameters and workspace (as the fused fits use them).
FitArgs fit_args(const phb_plan* plan, const phb_params* prm, void* ws, const int32_t* perm_out,
                 double* dudt, double* grad, double* hess, int32_t* fit_status,
                 int32_t* status_word);

// FP64 fused fit over all slots (list == null) or over list[0 .. *list_len);
// routed: the list is the FP32-mixed kernel's route queue (fit status 2).
cudaError_t launch_fit_fp64(const FitArgs& a, FitMode mode, const int32_t* list,
                            const int32_t* list_len, cudaStream_t st, bool routed = false);
int num_sms();
size_t l2_bytes();  // L2 cache size of the current device (queried once)

// Launch bookkeeping (measurement helpers, see include/phurbas_bench.h).
void note_launch(int count = 1);
// Bracket a fused-fit launch with the next traced event pair (if armed).
int trace_begin(int kernel_id, cudaStream_t st);
void trace_end(int slot, cudaStream_t st);

// Fused FP32-mixed / FP64 right-hand side of the slots marked 1 in the
// workspace's active-subset marks (R_AFLAG, n + 1 entries, the last 0), over
// the slot-order state already in the workspace; dudt in caller order at the
// marked particles only.
cudaError_t run_fit_marked(const phb_plan* plan, const phb_params* prm, void* ws, double* dudt,
                           int32_t* fit_status, int32_t* status_word, cudaStream_t st);

// Run the fused fit over the slot-order state already in the workspace:
// mixed kernel + FP64 queue, or the FP64 kernel alone; over all slots, or
// over list[0 .. *list_len) (list_cap entries at most) when list is given.
cudaError_t run_fit(const phb_plan* plan, const phb_params* prm, void* ws, FitMode mode,
                    const int32_t* perm_out, double* dudt, double* grad, double* hess,
                    int32_t* fit_status, int32_t* status_word, cudaStream_t st,
                    const int32_t* list = nullptr, const int32_t* list_len = nullptr,
                    int64_t list_cap = 0, const HostU* hu = nullptr);

}  // namespace phb
