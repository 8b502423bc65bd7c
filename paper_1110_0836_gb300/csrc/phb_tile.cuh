// Tiles: runs of `tile` consecutive particles in cell (slot) order.  Because
// cells are ordered brick by brick along a Hilbert curve, a tile covers a
// compact set of cells.  Its neighbourhood - the union of the reach boxes of
// its particles' cells, marked in a bitmap over the dilated bounding box - is
// planned once per neighbour build (the compaction kernel records the slot of
// every staged index) and staged in shared memory by every fused fit, so the
// fit's per-neighbour loads are shared-memory loads.  The staging order
// (marked cells in x-major box order, particles of a cell in slot order)
// defines the 16-bit tile-local neighbour indices of the lists.
//
// A tile whose bounding box holds more than kBoxCap cells, whose
// neighbourhood has more than kMarkCap cells or more than stage_cap particles
// "falls back": its kernels read neighbours from global memory through the
// global slot indices instead.
#pragma once

#include "phb_internal.cuh"

namespace phb {

constexpr int kBoxCap = 4096;   // cells of a tile's dilated bounding box (bitmap size)
constexpr int kBoxWords = kBoxCap / 32;
constexpr int kMarkCap = 1536;  // cells of the staged neighbourhood

struct TileShared {
  int cmin[3], cmax[3], rmax[3];
  int lo[3], dim[3];
  int boxcells;
  int ncells;    // marked (staged) cells
  int total;     // staged particles
  int fallback;  // 1: use global gathers for this tile
};

// Shared-memory arrays of a tile plan.
struct TileArrays {
  unsigned* bits;  // [kBoxWords] cells within reach of some tile particle
  int* wpre;       // [kBoxWords] marked cells before each bitmap word
  int* base;       // [kMarkCap + 1] first staged index of each marked cell
  int* cstart;     // [kMarkCap] first slot of each marked cell
  int* warp_tmp;   // [T / 32 + 1]
};

// Cells of reach of list radius r on axis a (covers every neighbour; see
// the cell-size argument in the neighbour search).
__device__ __forceinline__ int reach_cells(const Grid& g, int a, double r) {
  return static_cast<int>(ceil(r * g.inv_cell[a] * (1.0 + 1e-6)));
}

// Box coordinate (0 .. dim-1) of global cell c on axis a.
__device__ __forceinline__ int box_coord(const Grid& g, const TileShared& ts, int a, int c) {
  int d = c - ts.lo[a];
  if (g.periodic[a]) {
    const int nc = g.ncell[a];
    if (d < 0) d += nc;
    else if (d >= nc) d -= nc;
    if (static_cast<unsigned>(d) >= static_cast<unsigned>(nc)) {  // only for reaches beyond a box length
      d %= nc;
      if (d < 0) d += nc;
    }
  }
  return d;
}

__device__ __forceinline__ int wrap_cell(const Grid& g, int a, int c) {
  const int nc = g.ncell[a];
  if (g.periodic[a]) {
    c %= nc;
    if (c < 0) c += nc;
  }
  return c;
}

// Block-wide exclusive scan of v[0..m) in place (T threads); returns the total.
template <int T>
__device__ int block_scan_excl(int* v, int m, int* warp_tmp) {
  const int per = (m + T - 1) / T;
  const int b = threadIdx.x * per;
  int run = 0;
  for (int k = 0; k < per; ++k)
    if (b + k < m) run += v[b + k];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int inc = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) warp_tmp[wid] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int w = 0; w < T / 32; ++w) {
      const int x = warp_tmp[w];
      warp_tmp[w] = acc;
      acc += x;
    }
    warp_tmp[T / 32] = acc;
  }
  __syncthreads();
  int pre = inc - run + warp_tmp[wid];
  for (int k = 0; k < per; ++k)
    if (b + k < m) {
      const int x = v[b + k];
      v[b + k] = pre;
      pre += x;
    }
  const int total = warp_tmp[T / 32];
  __syncthreads();
  return total;
}

// Compact index of the marked box cell k (requires bit k set).
__device__ __forceinline__ int marked_index(const TileArrays& ta, int k) {
  const unsigned w = ta.bits[k >> 5];
  return ta.wpre[k >> 5] + __popc(w & ((1u << (k & 31)) - 1u));
}

// Plan the staging of tile [s0, s0 + cnt).  All T threads call it.  The
// staged neighbourhood is the union of the reach boxes of the tile's
// particles (exact, not the bounding box).  On return (if !ts.fallback)
// marked cell j holds staged indices [base[j], base[j+1]) starting at slot
// cstart[j]; box cell k maps to j by marked_index.  cellc: packed cell
// coordinates per slot; clin: (first slot, count) per linear cell index.
template <int T>
__device__ void tile_plan(const Grid& g, int s0, int cnt, const int32_t* __restrict__ cellc,
                          const double* __restrict__ slam, const int2* __restrict__ clin,
                          TileShared& ts, const TileArrays& ta) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int a = 0; a < 3; ++a) {
      ts.cmin[a] = 1 << 30;
      ts.cmax[a] = -1;
      ts.rmax[a] = 0;
    }
  }
  for (int w = tid; w < kBoxWords; w += T) ta.bits[w] = 0u;
  __syncthreads();
  int c[3] = {0, 0, 0}, R[3] = {0, 0, 0};
  if (tid < cnt) {
    unpack_cell(cellc[s0 + tid], c[0], c[1], c[2]);
    const double r = list_radius(g, slam[s0 + tid]);
    for (int a = 0; a < 3; ++a) {
      R[a] = reach_cells(g, a, r);
      atomicMin(&ts.cmin[a], c[a]);
      atomicMax(&ts.cmax[a], c[a]);
      atomicMax(&ts.rmax[a], R[a]);
    }
  }
  __syncthreads();
  if (tid == 0) {
    long long cells = 1;
    for (int a = 0; a < 3; ++a) {
      int lo = ts.cmin[a] - ts.rmax[a], hi = ts.cmax[a] + ts.rmax[a];
      if (g.periodic[a]) {
        if (hi - lo + 1 > g.ncell[a]) hi = lo + g.ncell[a] - 1;
      } else {
        lo = lo < 0 ? 0 : lo;
        hi = hi >= g.ncell[a] ? g.ncell[a] - 1 : hi;
      }
      ts.lo[a] = lo;
      ts.dim[a] = hi - lo + 1;
      cells *= ts.dim[a];
    }
    ts.boxcells = cells > kBoxCap ? kBoxCap : static_cast<int>(cells);
    ts.fallback = cells > kBoxCap ? 1 : 0;
  }
  __syncthreads();
  if (ts.fallback) return;
  // a particle in the same cell as the previous slot, with the same reach,
  // marks nothing new (cells hold consecutive slots)
  const int32_t pc = tid < cnt ? cellc[s0 + tid] : -1;
  const int pr = R[0] | (R[1] << 10) | (R[2] << 20);
  const int32_t prev_c = __shfl_up_sync(0xffffffffu, pc, 1);
  const int prev_r = __shfl_up_sync(0xffffffffu, pr, 1);
  const bool dup = (tid & 31) > 0 && prev_c == pc && prev_r == pr;
  // mark the reach box of every particle (whole axis where the reach wraps),
  // one masked atomicOr per run of cells along z
  if (tid < cnt && !dup) {
    int n3[3], st[3];
    for (int a = 0; a < 3; ++a) {
      if (g.periodic[a] && 2 * R[a] + 1 > g.ncell[a]) {
        st[a] = 0;
        n3[a] = g.ncell[a];
      } else {
        st[a] = c[a] - R[a];
        n3[a] = 2 * R[a] + 1;
      }
    }
    // z-run in box coordinates: [z0, z0 + nz) possibly split by the periodic wrap
    int zr0[2], zrn[2], nruns = 0;
    {
      int z0 = st[2], nz = n3[2];
      if (!g.periodic[2]) {
        const int a0 = z0 < 0 ? 0 : z0, a1 = z0 + nz > g.ncell[2] ? g.ncell[2] : z0 + nz;
        z0 = a0;
        nz = a1 - a0;
      }
      if (nz > 0) {
        const int b0 = box_coord(g, ts, 2, z0);
        const int first = b0 + nz <= ts.dim[2] ? nz : ts.dim[2] - b0;
        zr0[nruns] = b0;
        zrn[nruns++] = first;
        if (first < nz) {
          zr0[nruns] = 0;
          zrn[nruns++] = nz - first;
        }
      }
    }
    for (int ix = 0; ix < n3[0]; ++ix) {
      const int cx = st[0] + ix;
      if (!g.periodic[0] && (cx < 0 || cx >= g.ncell[0])) continue;
      const int bx = box_coord(g, ts, 0, cx);
      for (int iy = 0; iy < n3[1]; ++iy) {
        const int cy = st[1] + iy;
        if (!g.periodic[1] && (cy < 0 || cy >= g.ncell[1])) continue;
        const int row = (bx * ts.dim[1] + box_coord(g, ts, 1, cy)) * ts.dim[2];
        for (int q = 0; q < nruns; ++q) {
          int k = row + zr0[q], left = zrn[q];
          while (left > 0) {
            const int bit = k & 31, take = left < 32 - bit ? left : 32 - bit;
            const unsigned mask = (take == 32 ? 0xffffffffu : ((1u << take) - 1u)) << bit;
            atomicOr(&ta.bits[k >> 5], mask);
            k += take;
            left -= take;
          }
        }
      }
    }
  }
  __syncthreads();
  // marked cells per word -> word prefix
  const int nw = (ts.boxcells + 31) >> 5;
  for (int w = tid; w < nw; w += T) ta.wpre[w] = __popc(ta.bits[w]);
  __syncthreads();
  const int ncells = block_scan_excl<T>(ta.wpre, nw, ta.warp_tmp);
  if (tid == 0) {
    ts.ncells = ncells;
    if (ncells > kMarkCap) ts.fallback = 1;
  }
  __syncthreads();
  if (ts.fallback) return;
  // (first slot, count) of every marked cell, in box order: a thread per box
  // cell, so that the cell-table loads of a tile are issued in parallel
  const int d1 = ts.dim[1], d2 = ts.dim[2];
  for (int k = tid; k < ts.boxcells; k += T) {
    if (!(ta.bits[k >> 5] >> (k & 31) & 1u)) continue;
    const int j = marked_index(ta, k);
    const int bx = k / (d1 * d2), rr = k - bx * d1 * d2, by = rr / d2, bz = rr - by * d2;
    const int cx = wrap_cell(g, 0, ts.lo[0] + bx);
    const int cy = wrap_cell(g, 1, ts.lo[1] + by);
    const int cz = wrap_cell(g, 2, ts.lo[2] + bz);
    const int2 sc = clin[(static_cast<int64_t>(cx) * g.ncell[1] + cy) * g.ncell[2] + cz];
    ta.cstart[j] = sc.x;
    ta.base[j] = sc.y;
  }
  __syncthreads();
  const int total = block_scan_excl<T>(ta.base, ncells, ta.warp_tmp);
  if (tid == 0) {
    ta.base[ncells] = total;
    ts.total = total;
    if (total > g.stage_cap) ts.fallback = 1;
  }
  __syncthreads();
}

// Box index of the cell of a particle with packed cell p (always marked for a
// tile particle).
__device__ __forceinline__ int box_index(const Grid& g, const TileShared& ts, int32_t p) {
  int c[3];
  unpack_cell(p, c[0], c[1], c[2]);
  return (box_coord(g, ts, 0, c[0]) * ts.dim[1] + box_coord(g, ts, 1, c[1])) * ts.dim[2] +
         box_coord(g, ts, 2, c[2]);
}

}  // namespace phb
