// Cell binning (counting sort, stable by caller index) and the fixed-radius
// neighbour search of Paper II Sec. 2 / Sec. 2.1: strict, not mutual, radius
// of the gathering particle, no iteration.
//
// The search screens candidates in FP32 and decides the band of ambiguous
// candidates with the exact FP64 test, so every set equals the definition
// ((dx*dx + dy*dy) + dz*dz) < r*r evaluated in FP64 without contraction.
#include "phb_internal.cuh"
#include "phb_tile.cuh"

namespace phb {
namespace {

constexpr int kThreads = 256;
constexpr int kOwnerCap = 8192;  // list entries of a tile mapped to their particle in shared memory

inline unsigned blocks_for(int64_t n, int t = kThreads) { return static_cast<unsigned>((n + t - 1) / t); }

__global__ void k_keys(Grid g, const double* __restrict__ pos, const double* __restrict__ lam,
                       int32_t* __restrict__ keys, int32_t* __restrict__ counts,
                       int32_t* status_word) {
  const int n = g.n;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c[3];
  bool finite = true;
  for (int a = 0; a < 3; ++a) {
    const double x = pos[a * n + i];
    const bool f = finite64(x);
    finite &= f;
    c[a] = f ? cell_coord(g, a, x) : 0;
  }
  const double l = lam[i];
  if (!finite || !finite64(l)) raise_flag(status_word, PHB_FLAG_NONFINITE);
  if (!lambda_in_range(g, l)) raise_flag(status_word, PHB_FLAG_LAMBDA_RANGE);
  const int32_t k = cell_key(g, c[0], c[1], c[2]);
  keys[i] = k;
  atomicAdd(&counts[k], 1);
}

__global__ void k_scatter(int n, const int32_t* __restrict__ keys, const int32_t* __restrict__ cell_start,
                          int32_t* __restrict__ cursor, int32_t* __restrict__ perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t k = keys[i];
  perm[cell_start[k] + atomicAdd(&cursor[k], 1)] = i;
}

// Make the order inside each cell deterministic: ascending caller index.
// Thread per particle: its rank among the particles of its cell is the number
// of them with a smaller caller index (the cells' members come from the
// atomic scatter in arbitrary order).
__global__ void k_rank_cells(int n, const int32_t* __restrict__ keys,
                             const int32_t* __restrict__ cell_start,
                             const int32_t* __restrict__ scattered, int32_t* __restrict__ perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t k = keys[i];
  const int a = cell_start[k], b = cell_start[k + 1];
  int rank = 0;
  for (int t = a; t < b; ++t) rank += scattered[t] < i ? 1 : 0;
  perm[a + rank] = i;
}

// Slot-order copies of positions and lambda, the inverse permutation and the
// wrapped FP32 screen positions (wrapped by the same count as the cell).
__global__ void k_gather_pos(Grid g, const int32_t* __restrict__ perm, const double* __restrict__ pos,
                             const double* __restrict__ lam, int32_t* __restrict__ inv,
                             double* __restrict__ spos, double* __restrict__ slam,
                             float4* __restrict__ scr, int32_t* __restrict__ cellc) {
  const int n = g.n;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int i = perm[s];
  inv[i] = s;
  float w[3];
  int c[3];
  for (int a = 0; a < 3; ++a) {
    const double x = pos[a * n + i];
    spos[a * n + s] = x;
    double k = 0.0;
    bool kz = true;
    c[a] = finite64(x) ? cell_wrap(g, a, x, k, kz) : 0;
    w[a] = wrapped32(g, a, x, k, kz);
  }
  slam[s] = lam[i];
  scr[s] = make_float4(w[0], w[1], w[2], 0.f);
  cellc[s] = pack_cell(c[0], c[1], c[2]);
}

// (first slot, count) of every cell by linear index, for the tile planner and
// the search; the counts also go to lcnt[k] (lcnt[total] = 0), whose
// exclusive scan places the cells in linear order for the run search.
__global__ void k_cell_lin(Grid g, const int32_t* __restrict__ cell_start, int2* __restrict__ clin,
                           int32_t* __restrict__ lcnt, int32_t* __restrict__ misc) {
  const int64_t total = static_cast<int64_t>(g.ncell[0]) * g.ncell[1] * g.ncell[2];
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k == total) {
    lcnt[k] = 0;
    misc[1] = 0;  // the compaction's count of unstaged tiles
  }
  if (k >= total) return;
  const int cz = static_cast<int>(k % g.ncell[2]);
  const int cy = static_cast<int>((k / g.ncell[2]) % g.ncell[1]);
  const int cx = static_cast<int>(k / (static_cast<int64_t>(g.ncell[2]) * g.ncell[1]));
  const int32_t key = cell_key(g, cx, cy, cz);
  const int a = cell_start[key];
  clin[k] = make_int2(a, cell_start[key + 1] - a);
  lcnt[k] = cell_start[key + 1] - a;
}

// Screen records in linear cell order (z fastest; slot order inside a cell),
// with the slot in w, plus four padding records: the cells of one (x, y) row
// of a reach box are then one contiguous run.  lstart: exclusive scan of the
// linear-order counts.
__global__ void k_fill_lin(Grid g, const int32_t* __restrict__ cellc, const int2* __restrict__ clin,
                           const int32_t* __restrict__ lstart, const float4* __restrict__ scr,
                           float4* __restrict__ lscr) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.n) return;
  int cx, cy, cz;
  unpack_cell(cellc[s], cx, cy, cz);
  const int64_t k = (static_cast<int64_t>(cx) * g.ncell[1] + cy) * g.ncell[2] + cz;
  const float4 o = scr[s];
  lscr[lstart[k] + (s - clin[k].x)] = make_float4(o.x, o.y, o.z, __int_as_float(s));
  if (s < 4) lscr[g.n + s] = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));  // batch padding
}

struct Reach {
  int start, count;
  bool wrap, open;
};

__device__ __forceinline__ Reach axis_reach_cells(const Grid& g, int a, int c, int R) {
  Reach q;
  q.open = !g.periodic[a];
  if (g.periodic[a] && 2 * R + 1 >= g.ncell[a]) {
    q.start = 0;
    q.count = g.ncell[a];
    q.wrap = false;
  } else {
    q.start = c - R;
    q.count = 2 * R + 1;
    q.wrap = g.periodic[a] != 0;
  }
  return q;
}

__device__ __forceinline__ Reach axis_reach(const Grid& g, int a, int c, double r) {
  return axis_reach_cells(g, a, c, reach_cells(g, a, r));
}

__device__ __forceinline__ int axis_cell(const Grid& g, int a, const Reach& q, int k, bool& ok) {
  int c = q.start + k;
  ok = true;
  if (q.wrap) {
    int nc = g.ncell[a];
    c = c < 0 ? c + nc : (c >= nc ? c - nc : c);
  } else if (q.open && (c < 0 || c >= g.ncell[a])) {
    ok = false;
  }
  return c;
}

// Screen of candidate t against particle s: FP32 offsets of the wrapped
// positions and squared distance against the inner / outer screen radii;
// the exact FP64 test decides the ambiguous band.  kWrap = false skips the
// minimum image, which is then the identity (see the caller).
struct Screen {
  float in2, out2;
  double r2;
  float lenf[3], invlf[3];
};

__device__ __forceinline__ Screen make_screen(const Grid& g, double r) {
  Screen q;
  q.r2 = __dmul_rn(r, r);
  const double m = static_cast<double>(g.screen_margin) + 4e-7 * r;
  q.in2 = static_cast<float>(r > m ? (r - m) * (r - m) : 0.0);
  q.out2 = static_cast<float>((r + m) * (r + m));
  for (int a = 0; a < 3; ++a) {
    q.lenf[a] = g.lenf[a];
    q.invlf[a] = g.inv_lenf[a];  // formed on the host: no FP64 division per particle
  }
  return q;
}

// FP32 screen distance squared (the same arithmetic as is_neighbour): below
// q.in2 a neighbour, above q.out2 not, in between the exact test decides.
template <bool kWrap>
__device__ __forceinline__ float screen_d2(const Screen& q, float4 me, float4 o) {
  float dx = o.x - me.x, dy = o.y - me.y, dz = o.z - me.z;
  if (kWrap) {
    dx = fmaf(-q.lenf[0], rintf(dx * q.invlf[0]), dx);
    dy = fmaf(-q.lenf[1], rintf(dy * q.invlf[1]), dy);
    dz = fmaf(-q.lenf[2], rintf(dz * q.invlf[2]), dz);
  }
  return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

template <bool kWrap>
__device__ __forceinline__ bool is_neighbour(const Grid& g, const Screen& q, const double* spos,
                                             int s, int t, float4 me, float4 o) {
  float dx = o.x - me.x, dy = o.y - me.y, dz = o.z - me.z;
  if (kWrap) {
    dx = fmaf(-q.lenf[0], rintf(dx * q.invlf[0]), dx);
    dy = fmaf(-q.lenf[1], rintf(dy * q.invlf[1]), dy);
    dz = fmaf(-q.lenf[2], rintf(dz * q.invlf[2]), dz);
  }
  const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  if (d2 < q.in2) return true;
  if (d2 > q.out2) return false;
  return dist2_exact(g, spos, g.n, s, t) < q.r2;
}

// Whether every cell of the reach on axis a lies inside the grid without
// wrapping and spans less than half the box, so that the plain difference of
// two wrapped positions is already the minimum image: |dx| < (R + 1) cells
// <= len / 2 gives rint(dx / len) = 0.
__device__ __forceinline__ bool plain_axis(const Grid& g, int a, int c, const Reach& q) {
  if (!g.periodic[a]) return true;
  const int R = q.count / 2;
  return q.wrap && c - R >= 0 && c + R < g.ncell[a] && 2 * R + 3 <= g.ncell[a];
}

enum SearchOut { kCount = 0, kFillCsr = 1, kFillEll = 2 };

// Cell culling for the cell-by-cell search of reaches that cover a whole
// periodic axis (the run search does not cull): the reach box of 2R+1 cells
// per axis is cut to the cells that can hold a point within r of the
// particle.  With f the particle's
// fractional position in its cell, the nearest point of the cell at offset i
// is (i - f) cells away for i > 0, (-i - 1 + f) for i < 0 and 0 for i = 0.
// Distances are taken with a margin of 1e-3 cells plus the screen margin, so
// that only cells that cannot hold a neighbour are skipped; an axis whose
// reach covers the whole periodic grid is not culled.
struct Cull {
  float f[3];      // fractional position in the cell, clamped to [0, 1]
  float cell[3];   // cell edges
  float rr;        // (r + margin)^2
  bool on[3];      // axis culled
};

__device__ __forceinline__ float cull_d(const Cull& k, int a, int i) {
  if (!k.on[a] || i == 0) return 0.f;
  const float d = i > 0 ? i - k.f[a] : -i - 1 + k.f[a];
  return d > 0.f ? d * k.cell[a] : 0.f;
}

__device__ __forceinline__ Cull make_cull(const Grid& g, const double* spos, int s, const int (&c)[3],
                                          const Reach& qx, const Reach& qy, const Reach& qz, double r) {
  Cull k;
  const Reach* q[3] = {&qx, &qy, &qz};
  double mc = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double u = (spos[a * g.n + s] - g.lo[a]) * g.inv_cell[a];
    const double f = g.periodic[a] ? u - floor(u) : u - c[a];
    k.f[a] = static_cast<float>(f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f));
    k.cell[a] = static_cast<float>(g.cell[a]);
    k.on[a] = !(g.periodic[a] && !q[a]->wrap);  // not the whole-axis reach
    mc = g.cell[a] > mc ? g.cell[a] : mc;
  }
  const double rm = r + 1e-3 * mc + static_cast<double>(g.screen_margin);
  k.rr = static_cast<float>(rm * rm);
  return k;
}

// One particle's list: candidates from the culled cells within reach, looked
// up through the linear (first slot, count) table, in cell order (x, y, z)
// and slot order inside a cell.  kCount only counts; kFillCsr writes entries
// [base, end) of the CSR lists; kFillEll writes the first g.ell entries to
// the slot's row of the single-pass scratch.  Returns the exact count.
template <int OUT, bool kWrap>
__device__ int search_one(const Grid& g, const int2* __restrict__ clin, const float4* __restrict__ scr,
                          const double* __restrict__ spos, const Screen& q, const Cull& cu,
                          const Reach& qx, const Reach& qy, const Reach& qz, int s, int64_t base,
                          int64_t end, int32_t* __restrict__ out) {
  const float4 me = scr[s];
  const int Rx = qx.count / 2, Ry = qy.count / 2, Rz = qz.count / 2;
  int count = 0;
  for (int kx = 0; kx < qx.count; ++kx) {
    bool okx;
    const int cx = axis_cell(g, 0, qx, kx, okx);
    if (!okx) continue;
    const float dx = cull_d(cu, 0, kx - Rx);
    const float rx = cu.rr - dx * dx;
    if (rx < 0.f) continue;
    for (int ky = 0; ky < qy.count; ++ky) {
      bool oky;
      const int cy = axis_cell(g, 1, qy, ky, oky);
      if (!oky) continue;
      const float dy = cull_d(cu, 1, ky - Ry);
      const float ry = rx - dy * dy;
      if (ry < 0.f) continue;
      // z cells within reach of this row
      int z0 = 0, z1 = qz.count - 1;
      if (cu.on[2]) {
        const float sz = sqrtf(ry) / cu.cell[2];
        const int hi = static_cast<int>(floorf(sz + cu.f[2]));
        const int lo = -static_cast<int>(floorf(sz + 1.f - cu.f[2]));
        z0 = max(0, lo + Rz);
        z1 = min(qz.count - 1, hi + Rz);
      }
      const int64_t row = (static_cast<int64_t>(cx) * g.ncell[1] + cy) * g.ncell[2];
      for (int kz = z0; kz <= z1; ++kz) {
        bool okz;
        const int cz = axis_cell(g, 2, qz, kz, okz);
        if (!okz) continue;
        const int2 sc = clin[row + cz];
        for (int t = sc.x; t < sc.x + sc.y; ++t) {
          if (t == s || !is_neighbour<kWrap>(g, q, spos, s, t, me, scr[t])) continue;
          if (OUT == kFillCsr) {
            const int64_t e = base + count;
            if (e < g.capacity && e < end) out[e] = t;
          } else if (OUT == kFillEll) {
            if (count < g.ell) out[count] = t;
          }
          ++count;
        }
      }
    }
  }
  return count;
}

// Candidate records in linear cell order (k_fill_lin) and the cells' starts.
struct Lin {
  const float4* __restrict__ rec;
  const int32_t* __restrict__ start;
};

// The same list as search_one (cells in x, y, z order of the reach box,
// slot order inside a cell), for reaches that do not cover a whole periodic
// axis: the z cells of one (x, y) row are read as one run of the linear-order
// records (two where the row wraps a periodic z boundary), four candidates
// per batch so that their loads overlap.  The reach box is not culled per
// particle: the particles of one cell then walk identical rows and runs, so a
// warp's lanes stay together (measured faster than culling, which skips ~20%
// of the candidates but leaves half the lanes idle).
template <int OUT, bool kWrap>
__device__ int search_runs(const Grid& g, const Lin& lin, const double* __restrict__ spos,
                           const Screen& q, const Reach& qx, const Reach& qy, const Reach& qz,
                           float4 me, int s, int64_t base, int64_t end, int32_t* __restrict__ out) {
  const int ncz = g.ncell[2];
  int count = 0;
  auto take = [&](int t) {
    if (OUT == kFillCsr) {
      const int64_t e = base + count;
      if (e < g.capacity && e < end) out[e] = t;
    } else if (OUT == kFillEll) {
      if (count < g.ell) out[count] = t;
    }
    ++count;
  };
  for (int kx = 0; kx < qx.count; ++kx) {
    bool okx;
    const int cx = axis_cell(g, 0, qx, kx, okx);
    if (!okx) continue;
    for (int ky = 0; ky < qy.count; ++ky) {
      bool oky;
      const int cy = axis_cell(g, 1, qy, ky, oky);
      if (!oky) continue;
      int za = qz.start, zb = qz.start + qz.count - 1;
      // up to two runs of cells [a0, b0], [a1, b1], in the order of the reach offsets
      int a0 = za, b0 = zb, a1 = 0, b1 = -1;
      if (!qz.wrap) {
        a0 = max(za, 0);
        b0 = min(zb, ncz - 1);
      } else if (za < 0) {  // wraps below: cells ncz + za .., then 0 .. zb
        a0 = za + ncz;
        b0 = zb < 0 ? zb + ncz : ncz - 1;
        b1 = zb < 0 ? -1 : zb;
      } else if (zb >= ncz) {  // wraps above: cells za .. ncz - 1, then 0 .. zb - ncz
        a0 = za < ncz ? za : za - ncz;
        b0 = za < ncz ? ncz - 1 : zb - ncz;
        b1 = za < ncz ? zb - ncz : -1;
      }
      const int nseg = (a0 <= b0 ? 1 : 0) + (a1 <= b1 ? 1 : 0);
      if (a0 > b0) { a0 = a1; b0 = b1; }
      const int64_t row = (static_cast<int64_t>(cx) * g.ncell[1] + cy) * ncz;
      for (int k = 0; k < nseg; ++k) {
        const int t0 = lin.start[row + (k == 0 ? a0 : a1)];
        const int t1 = lin.start[row + (k == 0 ? b0 : b1) + 1];
        // batches of four (the records array is padded by four, so a batch
        // may read past the run): the screen sets a hit bit (inside the
        // inner radius) or an ambiguous bit (inside the band), the exact FP64
        // test settles the rare ambiguous ones, hits are then taken in order
        for (int t = t0; t < t1; t += 4) {
          const float4* rp = lin.rec + t;
          const float4 o0 = rp[0], o1 = rp[1], o2 = rp[2], o3 = rp[3];
          const unsigned live = t1 - t >= 4 ? 0xfu : (1u << (t1 - t)) - 1u;
          const float d0 = screen_d2<kWrap>(q, me, o0), d1 = screen_d2<kWrap>(q, me, o1);
          const float d2 = screen_d2<kWrap>(q, me, o2), d3 = screen_d2<kWrap>(q, me, o3);
          const unsigned self = (__float_as_int(o0.w) == s ? 1u : 0u) | (__float_as_int(o1.w) == s ? 2u : 0u) |
                                (__float_as_int(o2.w) == s ? 4u : 0u) | (__float_as_int(o3.w) == s ? 8u : 0u);
          const unsigned in = (d0 < q.in2 ? 1u : 0u) | (d1 < q.in2 ? 2u : 0u) | (d2 < q.in2 ? 4u : 0u) |
                              (d3 < q.in2 ? 8u : 0u);
          const unsigned out = (d0 <= q.out2 ? 1u : 0u) | (d1 <= q.out2 ? 2u : 0u) |
                               (d2 <= q.out2 ? 4u : 0u) | (d3 <= q.out2 ? 8u : 0u);
          const unsigned keep = live & ~self;
          unsigned hit = in & keep;
          const unsigned amb = out & ~in & keep;
          if (amb) {
            if ((amb & 1u) && dist2_exact(g, spos, g.n, s, __float_as_int(o0.w)) < q.r2) hit |= 1u;
            if ((amb & 2u) && dist2_exact(g, spos, g.n, s, __float_as_int(o1.w)) < q.r2) hit |= 2u;
            if ((amb & 4u) && dist2_exact(g, spos, g.n, s, __float_as_int(o2.w)) < q.r2) hit |= 4u;
            if ((amb & 8u) && dist2_exact(g, spos, g.n, s, __float_as_int(o3.w)) < q.r2) hit |= 8u;
          }
          if (hit) {
            if (hit & 1u) take(__float_as_int(o0.w));
            if (hit & 2u) take(__float_as_int(o1.w));
            if (hit & 4u) take(__float_as_int(o2.w));
            if (hit & 8u) take(__float_as_int(o3.w));
          }
        }
      }
    }
  }
  return count;
}

template <int OUT>
__device__ int search_particle(const Grid& g, const int2* __restrict__ clin, const Lin& lin,
                               const int32_t* __restrict__ cellc, const float4* __restrict__ scr,
                               const double* __restrict__ spos, double r, int s, int64_t base,
                               int64_t end, int32_t* __restrict__ out) {
  const Screen q = make_screen(g, r);
  int c[3];
  unpack_cell(cellc[s], c[0], c[1], c[2]);
  const Reach qx = axis_reach(g, 0, c[0], r);
  const Reach qy = axis_reach(g, 1, c[1], r);
  const Reach qz = axis_reach(g, 2, c[2], r);
  const bool plain =
      plain_axis(g, 0, c[0], qx) && plain_axis(g, 1, c[1], qy) && plain_axis(g, 2, c[2], qz);
  // a periodic axis whose reach is the whole axis has no wrap flag
  const bool whole = (g.periodic[0] && !qx.wrap) || (g.periodic[1] && !qy.wrap) ||
                     (g.periodic[2] && !qz.wrap);
  if (!whole) {
    const float4 me = scr[s];
    if (plain) return search_runs<OUT, false>(g, lin, spos, q, qx, qy, qz, me, s, base, end, out);
    return search_runs<OUT, true>(g, lin, spos, q, qx, qy, qz, me, s, base, end, out);
  }
  // a reach covering a whole periodic axis: cell by cell, culled
  const Cull cu = make_cull(g, spos, s, c, qx, qy, qz, r);
  if (plain) return search_one<OUT, false>(g, clin, scr, spos, q, cu, qx, qy, qz, s, base, end, out);
  return search_one<OUT, true>(g, clin, scr, spos, q, cu, qx, qy, qz, s, base, end, out);
}

// The CSR fill of one list longer than the scratch rows (rare): kept out of
// line so that it does not weigh on the compaction kernel's registers.
__device__ __noinline__ void search_overflow(const Grid& g, const int2* __restrict__ clin, Lin lin,
                                             const int32_t* __restrict__ cellc,
                                             const float4* __restrict__ scr,
                                             const double* __restrict__ spos, double r, int s,
                                             int64_t base, int64_t end, int32_t* __restrict__ out) {
  search_particle<kFillCsr>(g, clin, lin, cellc, scr, spos, r, s, base, end, out);
}

constexpr int kRunCap = 128;  // candidate runs a warp records (a reach of 3 cells: at most 98)

// Per warp: the cell's particles being searched ("homes", 32 at a time, padded
// to a multiple of four with homes that hit nothing) and the runs of their
// common reach box.
struct __align__(16) SearchWarp {
  float nx[32], ny[32], nz[32];  // negated wrapped FP32 positions
  float in2[32], out2[32];       // inner / outer screen radius^2
  int slot[32];
  double r2[32];                 // list radius^2 (exact test)
  int32_t* row[32];              // the home's scratch row
  int run_t0[kRunCap];           // first linear-order record of each run
  int run_pre[kRunCap + 1];      // candidates before each run (the last: the total)
};
// the home arrays are read four at a time as 16-byte vectors
static_assert(offsetof(SearchWarp, nx) % 16 == 0 && offsetof(SearchWarp, ny) % 16 == 0 &&
                  offsetof(SearchWarp, nz) % 16 == 0 && offsetof(SearchWarp, in2) % 16 == 0 &&
                  offsetof(SearchWarp, out2) % 16 == 0 && offsetof(SearchWarp, slot) % 16 == 0,
              "vector-read arrays of SearchWarp must be 16-byte aligned");

__device__ __forceinline__ int warp_excl_scan(int v, int lane) {
  int x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  return x - v;
}

// Squared FP32 screen distances of candidate o to two homes (a, b): packed
// FP32x2, each half rounded as screen_d2 rounds it.
template <bool kWrap>
__device__ __forceinline__ float2 screen_d2_pair(const Grid& g, float4 o, float2 nx, float2 ny, float2 nz) {
  float2 dx = __fadd2_rn(make_float2(o.x, o.x), nx);
  float2 dy = __fadd2_rn(make_float2(o.y, o.y), ny);
  float2 dz = __fadd2_rn(make_float2(o.z, o.z), nz);
  if (kWrap) {
    const float2 kx = __fmul2_rn(dx, make_float2(g.inv_lenf[0], g.inv_lenf[0]));
    const float2 ky = __fmul2_rn(dy, make_float2(g.inv_lenf[1], g.inv_lenf[1]));
    const float2 kz = __fmul2_rn(dz, make_float2(g.inv_lenf[2], g.inv_lenf[2]));
    dx = __ffma2_rn(make_float2(-g.lenf[0], -g.lenf[0]), make_float2(rintf(kx.x), rintf(kx.y)), dx);
    dy = __ffma2_rn(make_float2(-g.lenf[1], -g.lenf[1]), make_float2(rintf(ky.x), rintf(ky.y)), dy);
    dz = __ffma2_rn(make_float2(-g.lenf[2], -g.lenf[2]), make_float2(rintf(kz.x), rintf(kz.y)), dz);
  }
  return __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
}

// The candidates of one chunk (one per lane) against every home of the warp,
// four homes per round (their loads and screens independent): a ballot per
// home gives its hits, appended to its scratch row (S.row) in lane order.
template <bool kWrap>
__device__ __forceinline__ void screen_chunk(const Grid& g, const double* __restrict__ spos,
                                             const SearchWarp& S, int mh4, float4 o, int lane,
                                             int& cnt) {
  const int t = __float_as_int(o.w);
  const unsigned bit = 1u << lane, lt = bit - 1u;
#pragma unroll 1
  for (int i = 0; i < mh4; i += 4) {
    const float4 X = *reinterpret_cast<const float4*>(S.nx + i);
    const float4 Y = *reinterpret_cast<const float4*>(S.ny + i);
    const float4 Z = *reinterpret_cast<const float4*>(S.nz + i);
    const float4 I2 = *reinterpret_cast<const float4*>(S.in2 + i);
    const float4 O2 = *reinterpret_cast<const float4*>(S.out2 + i);
    const int4 SL = *reinterpret_cast<const int4*>(S.slot + i);
    const float2 d01 = screen_d2_pair<kWrap>(g, o, make_float2(X.x, X.y), make_float2(Y.x, Y.y),
                                             make_float2(Z.x, Z.y));
    const float2 d23 = screen_d2_pair<kWrap>(g, o, make_float2(X.z, X.w), make_float2(Y.z, Y.w),
                                             make_float2(Z.z, Z.w));
    const float d[4] = {d01.x, d01.y, d23.x, d23.y};
    const float in2[4] = {I2.x, I2.y, I2.z, I2.w};
    const float out2[4] = {O2.x, O2.y, O2.z, O2.w};
    const int sl[4] = {SL.x, SL.y, SL.z, SL.w};
    unsigned hit[4];
    unsigned band = 0u;  // bit u: inside home u's band (the exact test decides)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool other = t != sl[u];
      hit[u] = __ballot_sync(0xffffffffu, other && d[u] < in2[u]);
      band |= (other && !(d[u] < in2[u]) && d[u] <= out2[u]) ? 1u << u : 0u;
    }
    if (__any_sync(0xffffffffu, band != 0u)) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        hit[u] |= __ballot_sync(0xffffffffu, ((band >> u) & 1u) &&
                                                 dist2_exact(g, spos, g.n, sl[u], t) < S.r2[i + u]);
    }
    if ((hit[0] | hit[1] | hit[2] | hit[3]) != 0u) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (hit[u] == 0u) continue;
        const int c = __shfl_sync(0xffffffffu, cnt, i + u);
        if (hit[u] & bit) {
          const int e = c + __popc(hit[u] & lt);
          if (e < g.ell) S.row[i + u][e] = t;
        }
        if (lane == i + u) cnt = c + __popc(hit[u]);
      }
    }
  }
}

// Single pass, cell-major, for sets of one lambda: one warp per cell of the
// linear order, its particles ("homes", 32 at a time) sharing one reach box.
// The homes share one candidate sequence, the runs of their reach box in
// the order of the particle-major search (rows in (x, y) offset order, the z
// cells of a row as one or two runs of the linear-order records, slot order
// inside a cell), taken 32 candidates per chunk, one per lane; each chunk is
// screened against every home and a ballot per home appends its hits in lane
// order, so every list equals the particle-major one.  Writes the exact list
// lengths and the first g.ell entries of the lists it takes; a cell whose
// homes differ in reach, or whose reach covers a whole periodic axis or has
// more runs than a warp records, keeps the -1 of ncnt for k_search_ell.
// (Where lambda varies the particle-major search alone is faster: sparse
// cells leave most of a warp's homes empty, and cells of mixed reach would
// send scattered particles to the second pass.)
// One warp per block, so that the block scheduler hands out single cells
// (32 resident per SM at 64 registers).
__global__ void __launch_bounds__(32, 32) k_search_cells(Grid g, Lin lin,
                                                     const double* __restrict__ spos,
                                                     const double* __restrict__ slam,
                                                     int32_t* __restrict__ ncnt,
                                                     int32_t* __restrict__ ell) {
  __shared__ SearchWarp S;
  const int lane = threadIdx.x;
  const int ncx = g.ncell[0], ncy = g.ncell[1], ncz = g.ncell[2];
  const int64_t k = blockIdx.x;
  if (k >= static_cast<int64_t>(ncx) * ncy * ncz) return;
  const int h0 = lin.start[k], h1 = lin.start[k + 1];
  const int cz = static_cast<int>(k % ncz);
  const int cy = static_cast<int>((k / ncz) % ncy);
  const int cx = static_cast<int>(k / (static_cast<int64_t>(ncz) * ncy));
  for (int g0 = h0; g0 < h1; g0 += 32) {
    const int mh = min(32, h1 - g0);
    const bool mine = lane < mh;
    float4 me = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
    if (mine) me = lin.rec[g0 + lane];
    const int s = __float_as_int(me.w);
    double r = 0.0;
    int R[3] = {0, 0, 0};
    if (mine) {
      r = list_radius(g, slam[s]);
      for (int a = 0; a < 3; ++a) R[a] = reach_cells(g, a, r);
    }
    int U[3];
    bool same = true;
    for (int a = 0; a < 3; ++a) {
      U[a] = __shfl_sync(0xffffffffu, R[a], 0);
      same = same && (!mine || R[a] == U[a]);
    }
    if (!__all_sync(0xffffffffu, same) || U[0] < 0 || U[1] < 0 || U[2] < 0) continue;
    const Reach qx = axis_reach_cells(g, 0, cx, U[0]);
    const Reach qy = axis_reach_cells(g, 1, cy, U[1]);
    const Reach qz = axis_reach_cells(g, 2, cz, U[2]);
    const bool whole = (g.periodic[0] && !qx.wrap) || (g.periodic[1] && !qy.wrap) ||
                       (g.periodic[2] && !qz.wrap);
    const int64_t nrow = static_cast<int64_t>(qx.count) * qy.count;
    if (whole || nrow > kRunCap) continue;
    // the runs of the reach box, 32 rows at a time
    int nrun = 0, total = 0;
    for (int j0 = 0; j0 < nrow; j0 += 32) {
      const int j = j0 + lane;
      int nr = 0, ta = 0, la = 0, tb = 0, lb = 0;
      if (j < nrow) {
        const int kx = j / qy.count, ky = j - kx * qy.count;
        bool okx, oky;
        const int rx = axis_cell(g, 0, qx, kx, okx);
        const int ry = axis_cell(g, 1, qy, ky, oky);
        if (okx && oky) {
          const int za = qz.start, zb = qz.start + qz.count - 1;
          int a0 = za, b0 = zb, a1 = 0, b1 = -1;
          if (!qz.wrap) {
            a0 = max(za, 0);
            b0 = min(zb, ncz - 1);
          } else if (za < 0) {
            a0 = za + ncz;
            b0 = zb < 0 ? zb + ncz : ncz - 1;
            b1 = zb < 0 ? -1 : zb;
          } else if (zb >= ncz) {
            a0 = za < ncz ? za : za - ncz;
            b0 = za < ncz ? ncz - 1 : zb - ncz;
            b1 = za < ncz ? zb - ncz : -1;
          }
          nr = (a0 <= b0 ? 1 : 0) + (a1 <= b1 ? 1 : 0);
          if (a0 > b0) { a0 = a1; b0 = b1; }
          const int64_t row = (static_cast<int64_t>(rx) * ncy + ry) * ncz;
          if (nr >= 1) {
            ta = lin.start[row + a0];
            la = lin.start[row + b0 + 1] - ta;
          }
          if (nr == 2) {
            tb = lin.start[row + a1];
            lb = lin.start[row + b1 + 1] - tb;
          }
        }
      }
      const int rpos = nrun + warp_excl_scan(nr, lane);
      const int cpos = total + warp_excl_scan(la + lb, lane);
      if (rpos + nr <= kRunCap) {
        if (nr >= 1) {
          S.run_t0[rpos] = ta;
          S.run_pre[rpos] = cpos;
        }
        if (nr == 2) {
          S.run_t0[rpos + 1] = tb;
          S.run_pre[rpos + 1] = cpos + la;
        }
      }
      nrun = __shfl_sync(0xffffffffu, rpos + nr, 31);
      total = __shfl_sync(0xffffffffu, cpos + la + lb, 31);
    }
    if (nrun > kRunCap) continue;
    const int mh4 = (mh + 3) & ~3;
    if (lane < mh4) {
      Screen q = make_screen(g, r);
      if (!mine) {  // padding: hits nothing
        q.in2 = -1.f;
        q.out2 = -1.f;
      }
      S.nx[lane] = -me.x;
      S.ny[lane] = -me.y;
      S.nz[lane] = -me.z;
      S.in2[lane] = q.in2;
      S.out2[lane] = q.out2;
      S.slot[lane] = mine ? s : -2;
      S.r2[lane] = q.r2;
      S.row[lane] = ell + static_cast<int64_t>(mine ? s : 0) * g.ell;
    }
    if (lane == 0) S.run_pre[nrun] = total;
    __syncwarp();
    // the plain difference is the minimum image for the whole reach box
    const bool plain = plain_axis(g, 0, cx, qx) && plain_axis(g, 1, cy, qy) && plain_axis(g, 2, cz, qz);
    int run = 0;  // the run holding the next chunk's first candidate
    // candidate v0 + lane (none past the end: a NaN record hits nothing)
    auto fetch = [&](int v0) {
      const int v = v0 + lane;
      float4 o = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, __int_as_float(-1));
      int rn = run;
      if (v < total) {
        while (S.run_pre[rn + 1] <= v) ++rn;
        o = lin.rec[S.run_t0[rn] + (v - S.run_pre[rn])];
      }
      run = __shfl_sync(0xffffffffu, rn, 31);
      return o;
    };
    int cnt = 0;  // lane i: the list length of home i so far
    float4 next = fetch(0);
    for (int v0 = 0; v0 < total; v0 += 32) {
      const float4 o = next;
      if (v0 + 32 < total) next = fetch(v0 + 32);  // one chunk ahead
      if (plain) {
        screen_chunk<false>(g, spos, S, mh4, o, lane, cnt);
      } else {
        screen_chunk<true>(g, spos, S, mh4, o, lane, cnt);
      }
    }
    if (mine) ncnt[s] = cnt;
    __syncwarp();  // the next group of homes rewrites the warp's records
  }
}

// Single pass, thread per particle (slot order): exact list lengths and the
// first g.ell entries of every list (after the cell-major search, left_only:
// of the lists it left, ncnt still -1).
__global__ void __launch_bounds__(kThreads, 4) k_search_ell(Grid g, const int2* __restrict__ clin,
                                                         Lin lin, const int32_t* __restrict__ cellc,
                                                         const float4* __restrict__ scr,
                                                         const double* __restrict__ spos,
                                                         const double* __restrict__ slam,
                                                         int32_t* __restrict__ ncnt,
                                                         int32_t* __restrict__ ell, bool left_only) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.n) return;
  if (s == g.n - 1) ncnt[g.n] = 0;  // the offsets scan's sentinel
  if (left_only && ncnt[s] >= 0) return;
  const double r = list_radius(g, slam[s]);
  ncnt[s] = search_particle<kFillEll>(g, clin, lin, cellc, scr, spos, r, s, 0, 0,
                                      ell + static_cast<int64_t>(s) * g.ell);
}

// One CTA per tile: move the tile's lists from the single-pass scratch into
// the CSR arrays (searching again, straight into CSR, for lists longer than
// the scratch rows), plan the tile's staged neighbourhood and record it for
// the fused fit - (staged count, unstaged flag), the slot of every staged
// index, each tile particle's own staged index - and map every list entry to
// its staged index.
template <int T>
__global__ void __launch_bounds__(T, 1152 / T) k_compact(Grid g, const int2* __restrict__ clin, Lin lin,
                                               const int32_t* __restrict__ cellc,
                                               const float4* __restrict__ scr,
                                               const double* __restrict__ spos,
                                               const double* __restrict__ slam,
                                               const int32_t* __restrict__ ncnt,
                                               const int32_t* __restrict__ ell,
                                               const int64_t* __restrict__ off,
                                               int32_t* __restrict__ idx, uint16_t* __restrict__ lidx,
                                               int2* __restrict__ tplan, int32_t* __restrict__ tslot,
                                               uint16_t* __restrict__ lself, uint8_t* __restrict__ tmap,
                                               int32_t* fallback_count, int32_t* status_word) {
  __shared__ TileShared ts;
  __shared__ unsigned bits[kBoxWords];
  __shared__ int wpre[kBoxWords];
  __shared__ int base[kMarkCap + 1];
  __shared__ int cstart[kMarkCap];
  __shared__ int warp_tmp[T / 32 + 1];
  __shared__ int64_t toff[T + 1];
  __shared__ int tlen[T];
  __shared__ uint8_t owner[kOwnerCap];
  const TileArrays tarr{bits, wpre, base, cstart, warp_tmp};
  const int n = g.n;
  const int tid = threadIdx.x;
  const int s0 = blockIdx.x * T;
  const int cnt = min(T, n - s0);
  for (int k = tid; k <= cnt; k += T) toff[k] = off[s0 + k];
  __syncthreads();
  // fit thread -> tile particle in descending list length (ties: slot order),
  // so that the lanes of a fit warp run loops of similar length
  tlen[tid] = tid < cnt ? static_cast<int>(toff[tid + 1] - toff[tid]) : -1;
  __syncthreads();
  {
    const int len = tlen[tid];
    int rank = 0;
    for (int j = 0; j < T; ++j) {
      const int c = tlen[j];
      rank += (c > len || (c == len && j < tid)) ? 1 : 0;
    }
    tmap[static_cast<int64_t>(blockIdx.x) * T + rank] = static_cast<uint8_t>(tid);
  }
  if (tid < cnt) {
    const int s = s0 + tid;
    if (toff[tid + 1] > g.capacity) raise_flag(status_word, PHB_FLAG_CAPACITY);
    if (ncnt[s] > g.ell)
      search_overflow(g, clin, lin, cellc, scr, spos, list_radius(g, slam[s]), s, toff[tid],
                                toff[tid + 1], idx);
  }
  tile_plan<T>(g, s0, cnt, cellc, slam, clin, ts, tarr);
  const bool staged = !ts.fallback;
  if (tid == 0) {
    tplan[blockIdx.x] = make_int2(staged ? ts.total : 0, staged ? 0 : 1);
    if (!staged) atomicAdd(fallback_count, 1);
  }
  if (staged) {
    int32_t* ts_out = tslot + static_cast<int64_t>(blockIdx.x) * g.stage_cap;
    for (int j = tid; j < ts.ncells; j += T) {
      const int l0 = base[j], m = base[j + 1] - l0, t0 = cstart[j];
      for (int q = 0; q < m; ++q) ts_out[l0 + q] = t0 + q;
    }
    if (tid < cnt) {
      const int s = s0 + tid;
      const int j = marked_index(tarr, box_index(g, ts, cellc[s]));
      lself[s] = static_cast<uint16_t>(base[j] + (s - cstart[j]));
    }
  }
  // the tile's entries [e0, e1) as one flat range over the block (each
  // entry's tile particle from a byte map, or a binary search of the offsets
  // when the tile has more entries than the map holds)
  const int64_t e0 = toff[0];
  const int64_t e1 = toff[cnt] < g.capacity ? toff[cnt] : g.capacity;
  const bool mapped = e1 - e0 <= kOwnerCap;
  if (mapped && tid < cnt) {
    const int64_t a = toff[tid], b = toff[tid + 1] < e1 ? toff[tid + 1] : e1;
    for (int64_t e = a; e < b; ++e) owner[e - e0] = static_cast<uint8_t>(tid);
  }
  __syncthreads();
  // four entries per thread per round, their loads issued together (the
  // list slot, then its cell) so that several global loads are in flight
  auto owner_of = [&](int64_t e) {
    if (mapped) return static_cast<int>(owner[e - e0]);
    int lo = 0, hi = cnt - 1;  // the last p with toff[p] <= e
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (toff[mid] <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
  };
  constexpr int kB = 4;
  for (int64_t eb = e0 + tid; eb < e1; eb += kB * T) {
    int t[kB], c[kB];
    bool ok[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int64_t e = eb + static_cast<int64_t>(u) * T;
      ok[u] = e < e1;
      t[u] = 0;
      if (ok[u]) {
        const int p = owner_of(e);
        t[u] = tlen[p] > g.ell ? idx[e] : ell[static_cast<int64_t>(s0 + p) * g.ell + (e - toff[p])];
      }
    }
#pragma unroll
    for (int u = 0; u < kB; ++u) c[u] = (ok[u] && staged) ? cellc[t[u]] : 0;
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      if (!ok[u]) continue;
      const int64_t e = eb + static_cast<int64_t>(u) * T;
      idx[e] = t[u];
      if (staged) {
        const int j = marked_index(tarr, box_index(g, ts, c[u]));
        lidx[e] = static_cast<uint16_t>(base[j] + (t[u] - cstart[j]));
      }
    }
  }
}

// Tile order for the fused fit's schedule 1: tiles grouped by cost class
// floor(log2(list entries + 1)), most expensive class first (longest
// processing time first keeps the tail of the launch short).  One CTA.
__global__ void __launch_bounds__(1024) k_tile_order(int n, int T, int ntiles, int64_t cap,
                                                     const int64_t* __restrict__ off,
                                                     int32_t* __restrict__ order) {
  __shared__ int hist[65], cursor[65];
  const int tid = threadIdx.x;
  if (tid < 65) hist[tid] = 0;
  __syncthreads();
  for (int t = tid; t < ntiles; t += blockDim.x) {
    const int s0 = t * T, s1 = min(s0 + T, n);
    const int64_t a = off[s0] < cap ? off[s0] : cap, b = off[s1] < cap ? off[s1] : cap;
    const int cls = 64 - __clzll(static_cast<unsigned long long>(b - a + 1));
    atomicAdd(&hist[cls], 1);
  }
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int c = 64; c >= 0; --c) {
      cursor[c] = acc;
      acc += hist[c];
    }
  }
  __syncthreads();
  for (int t = tid; t < ntiles; t += blockDim.x) {
    const int s0 = t * T, s1 = min(s0 + T, n);
    const int64_t a = off[s0] < cap ? off[s0] : cap, b = off[s1] < cap ? off[s1] : cap;
    const int cls = 64 - __clzll(static_cast<unsigned long long>(b - a + 1));
    order[atomicAdd(&cursor[cls], 1)] = t;
  }
}

// -------- particle adaptivity scan (voids on a 9^3 grid of test points,
// clumps of too-close particles; see phb_adapt_scan)

// Slot-order copies of positions and lambda and wrapped FP32 screen
// positions for positions that may have moved since the build (the cells
// and tile plans of the build are left alone).
__global__ void k_adapt_gather(Grid g, const int32_t* __restrict__ perm, const double* __restrict__ pos,
                               const double* __restrict__ lam, double* __restrict__ spos,
                               double* __restrict__ slam, float4* __restrict__ scr) {
  const int n = g.n;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int i = perm[s];
  float w[3];
  for (int a = 0; a < 3; ++a) {
    const double x = pos[a * n + i];
    spos[a * n + s] = x;
    double k = 0.0;
    bool kz = true;
    if (finite64(x)) cell_wrap(g, a, x, k, kz);
    w[a] = wrapped32(g, a, x, k, kz);
  }
  slam[s] = lam[i];
  scr[s] = make_float4(w[0], w[1], w[2], 0.f);
}

constexpr int kGrid = 9;                       // test points per axis
constexpr int kGridPts = kGrid * kGrid * kGrid;

// FP32 offset of record o from me, minimum image on periodic axes.
__device__ __forceinline__ float3 offset32(const Screen& q, float4 me, float4 o) {
  float dx = o.x - me.x, dy = o.y - me.y, dz = o.z - me.z;
  dx = fmaf(-q.lenf[0], rintf(dx * q.invlf[0]), dx);
  dy = fmaf(-q.lenf[1], rintf(dy * q.invlf[1]), dy);
  dz = fmaf(-q.lenf[2], rintf(dz * q.invlf[2]), dz);
  return make_float3(dx, dy, dz);
}

// Exact FP64 squared distance from neighbour t of slot s to the test point
// at offset (ox, oy, oz): ((ex*ex + ey*ey) + ez*ez), e = min-image(x_t - x_s) - o.
__device__ __forceinline__ double test_dist2(const Grid& g, const double* spos, int n, int s, int t,
                                             double ox, double oy, double oz) {
  const double ex = __dsub_rn(min_image64(__dsub_rn(spos[t], spos[s]), g.len[0], g.periodic[0]), ox);
  const double ey =
      __dsub_rn(min_image64(__dsub_rn(spos[n + t], spos[n + s]), g.len[1], g.periodic[1]), oy);
  const double ez =
      __dsub_rn(min_image64(__dsub_rn(spos[2 * n + t], spos[2 * n + s]), g.len[2], g.periodic[2]), oz);
  return __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
}

// Thread per slot.  Every FP64 quantity that decides an output is computed
// with single IEEE-rounded operations in the order of the definition; FP32
// screens with a margin only skip work whose outcome they prove.
__global__ void __launch_bounds__(128) k_adapt_scan(Grid g, const int32_t* __restrict__ perm,
                                                   const double* __restrict__ spos,
                                                   const double* __restrict__ slam,
                                                   const float4* __restrict__ scr,
                                                   const int64_t* __restrict__ off,
                                                   const int32_t* __restrict__ idx, double vf, double cf,
                                                   int32_t* void_count, int32_t* best, double* cand,
                                                   int32_t* clump) {
  // candidate test points: every grid point that can lie inside r_f - d_v for
  // some lambda (a superset; each particle applies the exact test), ascending
  __shared__ int16_t pts[kGridPts];
  __shared__ int npts;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const double q = (g.rf_factor - vf) / (0.25 * g.rf_factor);
    const double lim = q > 0.0 ? q * q * (1.0 + 1e-6) : -1.0;
    int base = 0;
    for (int k0 = 0; k0 < kGridPts; k0 += 32) {
      const int k = k0 + lane;
      bool in = false;
      if (k < kGridPts) {
        const int kx = k / 81 - 4, ky = (k / 9) % 9 - 4, kz = k % 9 - 4;
        in = static_cast<double>(kx * kx + ky * ky + kz * kz) <= lim;
      }
      const unsigned m = __ballot_sync(0xffffffffu, in);
      if (in) pts[base + __popc(m & ((1u << lane) - 1u))] = static_cast<int16_t>(k);
      base += __popc(m);
    }
    if (lane == 0) npts = base;
  }
  __syncthreads();
  const int n = g.n;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int64_t N = n;
  const double lam = slam[s];
  const double r = __dmul_rn(g.rf_factor, lam);
  const double r2 = __dmul_rn(r, r);
  const double h = __dmul_rn(r, 0.25);
  const double dv = __dmul_rn(vf, lam);
  const double dv2 = __dmul_rn(dv, dv);
  const double rin = __dsub_rn(r, dv);
  const double rin2 = __dmul_rn(rin, rin);
  const double dc = __dmul_rn(cf, lam);
  const double dc2 = __dmul_rn(dc, dc);
  const Screen q = make_screen(g, r);
  // FP32 screens: |d32 - d| is within the coordinate margin; offsets and
  // squares add a few ulps of r
  const double m = static_cast<double>(g.screen_margin) + 1e-6 * r;
  const float v_in2 = static_cast<float>(dv > m ? (dv - m) * (dv - m) : 0.0);
  const float v_out2 = static_cast<float>((dv + m) * (dv + m));
  const float c_in2 = static_cast<float>(dc > m ? (dc - m) * (dc - m) : 0.0);
  const float c_out2 = static_cast<float>((dc + m) * (dc + m));
  const float r_in2 = static_cast<float>(r > m ? (r - m) * (r - m) : 0.0);
  const float r_out2 = static_cast<float>((r + m) * (r + m));
  const float4 me = scr[s];
  const int me_caller = perm[s];
  const int64_t beg = off[s];
  const int64_t end = off[s + 1] < g.capacity ? off[s + 1] : g.capacity;

  // clumps: a neighbour with a smaller caller index closer than d_c
  int32_t cl = 0;
  for (int64_t e = beg; e < end && !cl; ++e) {
    const int t = idx[e];
    if (perm[t] >= me_caller) continue;
    const float3 d = offset32(q, me, scr[t]);
    const float dd = fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z));
    if (dd < c_in2) cl = 1;
    else if (dd <= c_out2 && dist2_exact(g, spos, n, s, t) < dc2) cl = 1;
  }

  // voids: test points not within d_v of the particle or a neighbour
  int32_t cnt = 0, bk = -1;
  double bclear = -1.0;
  for (int p = 0; p < npts; ++p) {
    const int k = pts[p];
    const int kx = k / 81 - 4, ky = (k / 9) % 9 - 4, kz = k % 9 - 4;
    const double ox = __dmul_rn(static_cast<double>(kx), h);
    const double oy = __dmul_rn(static_cast<double>(ky), h);
    const double oz = __dmul_rn(static_cast<double>(kz), h);
    const double o2 = __dadd_rn(__dadd_rn(__dmul_rn(ox, ox), __dmul_rn(oy, oy)), __dmul_rn(oz, oz));
    if (!(o2 < rin2)) continue;  // outside r_f - d_v
    if (o2 < dv2) continue;      // covered by the particle itself
    const float fx = static_cast<float>(ox), fy = static_cast<float>(oy), fz = static_cast<float>(oz);
    bool covered = false;
    for (int64_t e = beg; e < end && !covered; ++e) {
      const int t = idx[e];
      const float3 d = offset32(q, me, scr[t]);
      const float ex = d.x - fx, ey = d.y - fy, ez = d.z - fz;
      const float e2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
      if (e2 < v_in2) covered = true;
      else if (e2 <= v_out2 && test_dist2(g, spos, n, s, t, ox, oy, oz) < dv2) covered = true;
    }
    if (covered) continue;
    // uncovered: its clearance, the smallest exact squared distance over the
    // particle (o2) and its exact r_f set.  An FP32 pass finds the smallest
    // screened distance over the entries proved (or, in the band, tested) to
    // be in the r_f set; only entries within twice the screen error of it
    // can hold the exact minimum, and only those are evaluated in FP64.
    float min32 = static_cast<float>(o2);
    for (int64_t e = beg; e < end; ++e) {
      const int t = idx[e];
      const float3 d = offset32(q, me, scr[t]);
      const float dd = fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z));
      if (dd > r_out2 || (dd >= r_in2 && !(dist2_exact(g, spos, n, s, t) < r2))) continue;
      const float ex = d.x - fx, ey = d.y - fy, ez = d.z - fz;
      const float e2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
      min32 = e2 < min32 ? e2 : min32;
    }
    const double band = sqrt(static_cast<double>(min32)) + 2.0 * m;
    const float band2 = static_cast<float>(band * band);
    double clear = o2;
    for (int64_t e = beg; e < end; ++e) {
      const int t = idx[e];
      const float3 d = offset32(q, me, scr[t]);
      const float ex = d.x - fx, ey = d.y - fy, ez = d.z - fz;
      if (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) > band2) continue;
      if (!(dist2_exact(g, spos, n, s, t) < r2)) continue;  // a skin entry, not in N(i)
      const double e2 = test_dist2(g, spos, n, s, t, ox, oy, oz);
      clear = e2 < clear ? e2 : clear;
    }
    ++cnt;
    if (clear > bclear) {
      bclear = clear;
      bk = k;
    }
  }
  if (void_count) void_count[me_caller] = cnt;
  if (best) best[me_caller] = bk;
  if (clump) clump[me_caller] = cl;
  if (cand) {
    double c[3] = {0.0, 0.0, 0.0};
    if (bk >= 0) {
      const int kk[3] = {bk / 81 - 4, (bk / 9) % 9 - 4, bk % 9 - 4};
      for (int a = 0; a < 3; ++a) c[a] = __dadd_rn(spos[a * N + s], __dmul_rn(static_cast<double>(kk[a]), h));
    }
    for (int a = 0; a < 3; ++a) cand[a * N + me_caller] = c[a];
  }
}

// Deletion and creation flags (caller order) from a scan: wants = survives
// (no clump mark), has a void and its point lies inside the box on every open
// axis; keep = survives.
__global__ void k_apply_wants(Grid g, const int32_t* __restrict__ best, const double* __restrict__ cand,
                              const int32_t* __restrict__ clump, int32_t* __restrict__ wants,
                              int32_t* __restrict__ keep) {
  const int n = g.n;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  if (i == n) {  // scan sentinels
    keep[n] = 0;
    return;
  }
  const int64_t N = n;
  bool in = true;
  for (int a = 0; a < 3; ++a) {
    const double c = cand[a * N + i];
    if (!g.periodic[a]) in = in && c >= g.lo[a] && c < __dadd_rn(g.lo[a], g.len[a]);
  }
  keep[i] = clump[i] == 0 ? 1 : 0;
  wants[i] = (clump[i] == 0 && best[i] >= 0 && in) ? 1 : 0;
}

// create[i]: i wants a particle and no neighbour j of its exact r_f set with
// j < i wants one at a point closer than d_v = vf lambda_i (FP64, minimum
// image, in the order ((dx*dx + dy*dy) + dz*dz)).  Thread per slot.
__global__ void k_apply_create(Grid g, const int32_t* __restrict__ perm, const double* __restrict__ spos,
                               const double* __restrict__ slam, const int64_t* __restrict__ off,
                               const int32_t* __restrict__ idx, const double* __restrict__ cand,
                               const int32_t* __restrict__ wants, double vf,
                               int32_t* __restrict__ create) {
  const int n = g.n;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s > n) return;
  if (s == n) {
    create[n] = 0;
    return;
  }
  const int64_t N = n;
  const int i = perm[s];
  int32_t c = wants[i];
  if (c) {
    const double lam = slam[s];
    const double r = __dmul_rn(g.rf_factor, lam);
    const double r2 = __dmul_rn(r, r);
    const double dv = __dmul_rn(vf, lam);
    const double dv2 = __dmul_rn(dv, dv);
    const double ci[3] = {cand[i], cand[N + i], cand[2 * N + i]};
    const int64_t end = off[s + 1] < g.capacity ? off[s + 1] : g.capacity;
    for (int64_t e = off[s]; e < end && c; ++e) {
      const int t = idx[e];
      const int j = perm[t];
      if (j >= i || !wants[j]) continue;
      double dd[3];
      for (int a = 0; a < 3; ++a) dd[a] = min_image64(__dsub_rn(cand[a * N + j], ci[a]), g.len[a], g.periodic[a]);
      const double d2 =
          __dadd_rn(__dadd_rn(__dmul_rn(dd[0], dd[0]), __dmul_rn(dd[1], dd[1])), __dmul_rn(dd[2], dd[2]));
      if (!(d2 < dv2)) continue;
      if (dist2_exact(g, spos, n, s, t) < r2) c = 0;  // not a skin entry
    }
  }
  create[i] = c;
}

// Survivors (in order) then new particles (in parent order) into the output
// arrays of leading dimension cap; ks / cs: exclusive scans of keep / create
// (their totals at n).  New particles: lambda of the parent and its
// second-order Taylor value at o = c - x, accumulated as
// U + sum_a (g_a o_a + sum_b ((h_ab / 2) o_a) o_b).
__global__ void k_apply_write(int n, int64_t cap, const double* __restrict__ pos,
                              const double* __restrict__ lam, const double* __restrict__ U,
                              const double* __restrict__ cand, const double* __restrict__ grad,
                              const double* __restrict__ hess, const int32_t* __restrict__ ks,
                              const int32_t* __restrict__ cs, double* __restrict__ pos_out,
                              double* __restrict__ lam_out, double* __restrict__ U_out,
                              int64_t* __restrict__ origin, int64_t* m_out, int32_t* status_word) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t N = n;
  const int64_t nk = ks[n];
  if (i == 0) {
    const int64_t m = nk + cs[n];
    *m_out = m;
    if (m > cap) raise_flag(status_word, PHB_FLAG_CAPACITY);
  }
  if (ks[i + 1] != ks[i]) {
    const int64_t k = ks[i];
    if (k < cap) {
      for (int a = 0; a < 3; ++a) pos_out[a * cap + k] = pos[a * N + i];
      lam_out[k] = lam[i];
      for (int f = 0; f < 8; ++f) U_out[f * cap + k] = U[f * N + i];
      origin[k] = i;
    }
  }
  if (cs[i + 1] != cs[i]) {
    const int64_t k = nk + cs[i];
    if (k < cap) {
      double o[3];
      for (int a = 0; a < 3; ++a) {
        const double c = cand[a * N + i];
        pos_out[a * cap + k] = c;
        o[a] = __dsub_rn(c, pos[a * N + i]);
      }
      lam_out[k] = lam[i];
      const int hx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
      for (int f = 0; f < 8; ++f) {
        double u = U[f * N + i];
        for (int a = 0; a < 3; ++a) {
          u = __dadd_rn(u, __dmul_rn(grad[(f * 3 + a) * N + i], o[a]));
          for (int b = 0; b < 3; ++b)
            u = __dadd_rn(u, __dmul_rn(__dmul_rn(__dmul_rn(0.5, hess[(f * 6 + hx[a][b]) * N + i]), o[a]), o[b]));
        }
        U_out[f * cap + k] = u;
      }
      origin[k] = N + i;
    }
  }
}

// -------- storage order
__global__ void k_identity(int n, int32_t* __restrict__ perm, int32_t* __restrict__ inv) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  perm[s] = s;
  inv[s] = s;
}

// -------- export in caller numbering
__global__ void k_user_counts(int n, const int32_t* __restrict__ inv, const int64_t* __restrict__ off,
                              int32_t* __restrict__ ucnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  if (i == n) { ucnt[n] = 0; return; }
  const int s = inv[i];
  ucnt[i] = static_cast<int32_t>(off[s + 1] - off[s]);
}

__global__ void k_user_fill(int n, int64_t cap, const int32_t* __restrict__ inv,
                            const int32_t* __restrict__ perm, const int64_t* __restrict__ off,
                            const int32_t* __restrict__ idx, const int64_t* __restrict__ uoff,
                            int32_t* __restrict__ uidx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = inv[i];
  const int64_t a = off[s], b = off[s + 1] < cap ? off[s + 1] : cap;
  int32_t* v = uidx + uoff[i];
  const int m = static_cast<int>(b > a ? b - a : 0);
  for (int k = 0; k < m; ++k) v[k] = perm[idx[a + k]];
  for (int k = 1; k < m; ++k) {  // ascending caller index
    int32_t x = v[k];
    int j = k - 1;
    while (j >= 0 && v[j] > x) { v[j + 1] = v[j]; --j; }
    v[j + 1] = x;
  }
}

}  // namespace

cudaError_t build_neighbors_impl(const phb_plan* p, const double* pos, const double* lam, void* ws,
                                 int32_t* status_word, cudaStream_t st) {
  const Grid g = make_grid(p);
  const int n = g.n;
  int32_t* keys = region<int32_t>(p, ws, R_KEYS);
  int32_t* perm = region<int32_t>(p, ws, R_PERM);
  int32_t* inv = region<int32_t>(p, ws, R_INV);
  int32_t* cell = region<int32_t>(p, ws, R_CELL);
  int32_t* cursor = region<int32_t>(p, ws, R_CURSOR);
  int64_t* bsum = region<int64_t>(p, ws, R_SCAN);
  double* spos = region<double>(p, ws, R_SPOS);
  double* slam = region<double>(p, ws, R_SLAM);
  float4* scr = region<float4>(p, ws, R_SCREEN);
  int32_t* ncnt = region<int32_t>(p, ws, R_NCNT);
  int64_t* off = region<int64_t>(p, ws, R_OFF);
  int32_t* idx = region<int32_t>(p, ws, R_IDX);
  uint16_t* lidx = region<uint16_t>(p, ws, R_LIDX);
  int32_t* cellc = region<int32_t>(p, ws, R_CELLC);
  int2* clin = region<int2>(p, ws, R_CLIN);
  int32_t* misc = region<int32_t>(p, ws, R_MISC);
  cudaError_t e;
  // cell counts and scatter cursors are adjacent regions: one clear
  const size_t clear = p->ws_off[R_CURSOR] + p->nkeys * sizeof(int32_t) - p->ws_off[R_CELL];
  if ((e = cudaMemsetAsync(cell, 0, clear, st))) return e;
  k_keys<<<blocks_for(n), kThreads, 0, st>>>(g, pos, lam, keys, cell, status_word);
  note_launch();
  if ((e = scan_exclusive_i32(cell, p->nkeys + 1, bsum, st))) return e;
  // the inverse-permutation region (written later by k_gather_pos) holds the
  // scattered order until the ranking puts it into ascending caller index
  k_scatter<<<blocks_for(n), kThreads, 0, st>>>(n, keys, cell, cursor, inv);
  note_launch();
  k_rank_cells<<<blocks_for(n), kThreads, 0, st>>>(n, keys, cell, inv, perm);
  note_launch();
  k_gather_pos<<<blocks_for(n), kThreads, 0, st>>>(g, perm, pos, lam, inv, spos, slam, scr, cellc);
  note_launch();
  const int64_t ncells = int64_t(p->ncell[0]) * p->ncell[1] * p->ncell[2];
  int32_t* lstart = region<int32_t>(p, ws, R_LSTART);
  float4* lscr = region<float4>(p, ws, R_LSCR);
  k_cell_lin<<<blocks_for(ncells + 1), kThreads, 0, st>>>(g, cell, clin, lstart, misc);
  note_launch();
  if ((e = scan_exclusive_i32(lstart, ncells + 1, bsum, st))) return e;
  k_fill_lin<<<blocks_for(n), kThreads, 0, st>>>(g, cellc, clin, lstart, scr, lscr);
  note_launch();
  const Lin lin{lscr, lstart};
  int32_t* ell = region<int32_t>(p, ws, R_ELL);
  // one lambda: cell-major, then particle-major for the lists it left;
  // lambda varying: particle-major
  const bool cell_major = p->lambda_max <= 1.01 * p->lambda_min;
  if (cell_major && (e = cudaMemsetAsync(ncnt, 0xff, static_cast<size_t>(n) * sizeof(int32_t), st)))
    return e;
  int tr = trace_begin(4, st);
  if (cell_major) {
    k_search_cells<<<static_cast<unsigned>(ncells), 32, 0, st>>>(g, lin, spos, slam, ncnt, ell);
    note_launch();
  }
  k_search_ell<<<blocks_for(n), kThreads, 0, st>>>(g, clin, lin, cellc, scr, spos, slam, ncnt, ell,
                                                   cell_major);
  trace_end(tr, st);
  note_launch();
  if ((e = scan_exclusive_i32_to_i64(ncnt, off, n + 1, bsum, st))) return e;
  const unsigned tiles = static_cast<unsigned>(p->ntiles);
  int2* tplan = region<int2>(p, ws, R_TPLAN);
  int32_t* tslot = region<int32_t>(p, ws, R_TSLOT);
  uint16_t* lself = region<uint16_t>(p, ws, R_LSELF);
  uint8_t* tmap = region<uint8_t>(p, ws, R_TMAP);
  tr = trace_begin(5, st);
  // nine 128-thread blocks per SM at 56 registers: 2048 tiles in 1.5 waves
  // of 1368 instead of 1.7 of 1216 (the shared memory of nine needs the
  // largest carve-out)
  cudaFuncSetAttribute(k_compact<128>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(k_compact<64>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  if (p->tile == 128)
    k_compact<128><<<tiles, 128, 0, st>>>(g, clin, lin, cellc, scr, spos, slam, ncnt, ell, off, idx, lidx,
                                          tplan, tslot, lself, tmap, misc + 1, status_word);
  else
    k_compact<64><<<tiles, 64, 0, st>>>(g, clin, lin, cellc, scr, spos, slam, ncnt, ell, off, idx, lidx,
                                        tplan, tslot, lself, tmap, misc + 1, status_word);
  trace_end(tr, st);
  note_launch();
  if (p->schedule == 1) {  // only schedule 1 of the fit reads the tile order
    k_tile_order<<<1, 1024, 0, st>>>(n, p->tile, p->ntiles, p->nbr_capacity, off,
                                     region<int32_t>(p, ws, R_TORDER));
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t export_neighbors_impl(const phb_plan* p, const void* ws_c, int64_t* uoff, int32_t* uidx,
                                  cudaStream_t st) {
  void* ws = const_cast<void*>(ws_c);
  const int n = static_cast<int>(p->n);
  const int32_t* perm = region<int32_t>(p, ws, R_PERM);
  const int32_t* inv = region<int32_t>(p, ws, R_INV);
  const int64_t* off = region<int64_t>(p, ws, R_OFF);
  const int32_t* idx = region<int32_t>(p, ws, R_IDX);
  int32_t* ucnt = region<int32_t>(p, ws, R_QUEUE);  // scratch: n+1 fits before R_PC (>= n+64 ints)
  int64_t* bsum = region<int64_t>(p, ws, R_SCAN);
  cudaError_t e;
  k_user_counts<<<blocks_for(n + 1), kThreads, 0, st>>>(n, inv, off, ucnt);
  note_launch();
  if ((e = scan_exclusive_i32_to_i64(ucnt, uoff, n + 1, bsum, st))) return e;
  k_user_fill<<<blocks_for(n), kThreads, 0, st>>>(n, p->nbr_capacity, inv, perm, off, idx, uoff, uidx);
  note_launch();
  return cudaGetLastError();
}

}  // namespace phb

using namespace phb;

extern "C" phb_status phb_build_neighbors(const phb_plan* plan, const double* pos,
                                          const double* lambda, void* ws, size_t ws_bytes,
                                          int32_t* status_word, phb_stream_t stream) {
  phb_status s = check_common(plan, ws, ws_bytes, plan ? plan->ws_off[R_END_COMMON] : 0);
  if (s != PHB_OK) return s;
  if (!pos || !lambda) return PHB_ERR_INVALID_ARG;
  return launch_status(build_neighbors_impl(plan, pos, lambda, ws, status_word,
                                            reinterpret_cast<cudaStream_t>(stream)));
}

extern "C" phb_status phb_adapt_scan(const phb_plan* plan, const double* pos, const double* lambda,
                                     double void_factor, double clump_factor, void* ws, size_t ws_bytes,
                                     int32_t* void_count, int32_t* best, double* cand, int32_t* clump,
                                     int32_t* status_word, phb_stream_t stream) {
  phb_status s = check_common(plan, ws, ws_bytes, plan ? plan->ws_off[R_END_COMMON] : 0);
  if (s != PHB_OK) return s;
  if (!pos || !lambda) return PHB_ERR_INVALID_ARG;
  if (!(void_factor > 0.0) || !(void_factor < plan->rf_factor) || !(clump_factor >= 0.0) ||
      !(clump_factor < plan->rf_factor))
    return PHB_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Grid g = make_grid(plan);
  const int n = g.n;
  const int32_t* perm = region<int32_t>(plan, ws, R_PERM);
  double* spos = region<double>(plan, ws, R_SPOS);
  double* slam = region<double>(plan, ws, R_SLAM);
  float4* scr = region<float4>(plan, ws, R_SCREEN);
  k_adapt_gather<<<blocks_for(n), kThreads, 0, st>>>(g, perm, pos, lambda, spos, slam, scr);
  note_launch();
  k_adapt_scan<<<blocks_for(n, 128), 128, 0, st>>>(g, perm, spos, slam, scr,
                                                   region<int64_t>(plan, ws, R_OFF),
                                                   region<int32_t>(plan, ws, R_IDX), void_factor,
                                                   clump_factor, void_count, best, cand, clump);
  note_launch();
  return launch_status(cudaGetLastError());
}

extern "C" phb_status phb_adapt_apply(const phb_plan* plan, const double* pos, const double* lambda,
                                      const double* U, const int32_t* best, const double* cand,
                                      const int32_t* clump, const double* grad, const double* hess,
                                      double void_factor, int64_t cap, double* pos_out,
                                      double* lambda_out, double* U_out, int64_t* origin,
                                      int64_t* m_out, void* ws, size_t ws_bytes, int32_t* status_word,
                                      phb_stream_t stream) {
  phb_status s = check_common(plan, ws, ws_bytes, plan ? plan->ws_off[R_END_COMMON] : 0);
  if (s != PHB_OK) return s;
  if (!pos || !lambda || !U || !best || !cand || !clump || !grad || !hess || !pos_out ||
      !lambda_out || !U_out || !origin || !m_out || cap < 0)
    return PHB_ERR_INVALID_ARG;
  if (!(void_factor > 0.0) || !(void_factor < plan->rf_factor)) return PHB_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Grid g = make_grid(plan);
  const int n = g.n;
  const int32_t* perm = region<int32_t>(plan, ws, R_PERM);
  double* spos = region<double>(plan, ws, R_SPOS);
  double* slam = region<double>(plan, ws, R_SLAM);
  float4* scr = region<float4>(plan, ws, R_SCREEN);
  int32_t* wants = region<int32_t>(plan, ws, R_QUEUE);
  int32_t* keep = region<int32_t>(plan, ws, R_AFLAG);
  int32_t* create = region<int32_t>(plan, ws, R_ALIST);
  int64_t* bsum = region<int64_t>(plan, ws, R_SCAN);
  cudaError_t e;
  k_adapt_gather<<<blocks_for(n), kThreads, 0, st>>>(g, perm, pos, lambda, spos, slam, scr);
  note_launch();
  k_apply_wants<<<blocks_for(n + 1), kThreads, 0, st>>>(g, best, cand, clump, wants, keep);
  note_launch();
  k_apply_create<<<blocks_for(n + 1), kThreads, 0, st>>>(g, perm, spos, slam,
                                                         region<int64_t>(plan, ws, R_OFF),
                                                         region<int32_t>(plan, ws, R_IDX), cand, wants,
                                                         void_factor, create);
  note_launch();
  if ((e = scan_exclusive_i32(keep, n + 1, bsum, st))) return launch_status(e);
  if ((e = scan_exclusive_i32(create, n + 1, bsum, st))) return launch_status(e);
  k_apply_write<<<blocks_for(n), kThreads, 0, st>>>(n, cap, pos, lambda, U, cand, grad, hess, keep, create,
                                                    pos_out, lambda_out, U_out, origin, m_out,
                                                    status_word);
  note_launch();
  return launch_status(cudaGetLastError());
}

extern "C" phb_status phb_reorder(const phb_plan* plan, double* pos, double* lambda, double* U,
                                  int32_t* perm_out, void* ws, size_t ws_bytes, int32_t* status_word,
                                  phb_stream_t stream) {
  phb_status s = check_common(plan, ws, ws_bytes, plan ? plan->ws_off[R_END_COMMON] : 0);
  if (s != PHB_OK) return s;
  if (!pos || !lambda || !U) return PHB_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Grid g = make_grid(plan);
  const int64_t N = plan->n;
  int32_t* perm = region<int32_t>(plan, ws, R_PERM);
  cudaError_t e;
  // slot-order copies of all three arrays, then back over the caller's
  if ((e = gather_sorted(plan, g, pos, lambda, U, ws, status_word, st))) return launch_status(e);
  if (perm_out && (e = cudaMemcpyAsync(perm_out, perm, N * sizeof(int32_t), cudaMemcpyDeviceToDevice, st)))
    return launch_status(e);
  if ((e = cudaMemcpyAsync(pos, region<double>(plan, ws, R_SPOS), 3 * N * sizeof(double),
                           cudaMemcpyDeviceToDevice, st)))
    return launch_status(e);
  if ((e = cudaMemcpyAsync(lambda, region<double>(plan, ws, R_SLAM), N * sizeof(double),
                           cudaMemcpyDeviceToDevice, st)))
    return launch_status(e);
  if ((e = cudaMemcpyAsync(U, region<double>(plan, ws, R_SU), 8 * N * sizeof(double),
                           cudaMemcpyDeviceToDevice, st)))
    return launch_status(e);
  k_identity<<<blocks_for(N), kThreads, 0, st>>>(g.n, perm, region<int32_t>(plan, ws, R_INV));
  note_launch();
  return launch_status(cudaGetLastError());
}

extern "C" int64_t phb_neighbor_total(const phb_plan* plan, const void* ws, phb_stream_t stream) {
  if (!plan || !ws || plan->ws_bytes == 0) return -1;
  int64_t total = -1;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t* off = region<int64_t>(plan, ws, R_OFF);
  if (cudaMemcpyAsync(&total, off + plan->n, sizeof(int64_t), cudaMemcpyDeviceToHost, st) !=
      cudaSuccess)
    return -1;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
  return total;
}

extern "C" phb_status phb_export_neighbors(const phb_plan* plan, const void* ws, int64_t* off,
                                           int32_t* idx, int64_t idx_capacity, phb_stream_t stream) {
  if (!plan || !ws || !off || !idx || plan->ws_bytes == 0) return PHB_ERR_INVALID_ARG;
  // the export writes its counts into the route-queue region (n int32 + pad)
  int64_t total = phb_neighbor_total(plan, ws, stream);
  if (total < 0) return PHB_ERR_CUDA;
  if (total > idx_capacity || total > plan->nbr_capacity) return PHB_ERR_CAPACITY;
  return launch_status(export_neighbors_impl(plan, ws, off, idx, reinterpret_cast<cudaStream_t>(stream)));
}
