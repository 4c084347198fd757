// Cell-list neighbour search (the linked-cell list that replaces an O(N^2)
// pair search, paper Sec. "Massive Parallelism within Tinker-HP").
//
// Pipeline for a batch of systems, all on one stream, no host synchronisation:
//   k_init     zero counters, copy the per-system descriptors to the device
//   k_prep     per input atom: mask, validation, per-system / per-species counts,
//              bounding boxes (non-periodic systems)
//   k_setup    per system: cell grid, packed atom / cell offsets; 128-row padded
//              species segments of the AEV rows
//   k_bin      per atom: cell index, rank inside the cell, AEV row (slot)
//   k_scan     exclusive scan of the cell counts
//   k_scatter  packed (cell-ordered) float4 coordinates and index maps
//   k_neighbors one CTA per home cell: the atoms of the 27 neighbour cells are
//              staged in shared memory, sorted by species, and listed per
//              octant of the home cell (the candidates near that octant's
//              atoms); one warp per centre scans its octant's list, keeps pairs
//              with R <= rc_r, marks R <= rc_a and writes species-sorted lists
//              (per-centre search from global memory when a neighbourhood does
//              not fit the stage)
// A one-chunk batch of at most 2048 atoms runs init .. scatter as one CTA
// (k_front).  With a Verlet skin, k_skin_check measures the displacement since
// the last build, the front-end kernels and k_neighbors return at once when no
// rebuild is due, and k_list_refresh cuts the lists at Rc + skin down to the
// cutoffs on every call.
#include <algorithm>

#include "nnp_internal.cuh"

namespace nnp {

namespace {

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ int find_sys(const BatchParams& bp, int idx) {
  // last system whose in_base <= idx (in_base relative to the chunk start)
  int lo = 0, hi = bp.n_sys - 1;
  const int base0 = bp.sys[0].in_base;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (bp.sys[mid].in_base - base0 <= idx) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void init_body(const Ws& ws, const BatchParams& bp, int zero_all,
                                          int n_in, int tid, int stride) {
  const bool rebuild = lists_rebuild(ws);
  // the AEV kernel ORs this call's live slices into the tile masks
  if (zero_all && ws.tile_mask)
    for (int i = tid; i <= ws.row_cap / 128; i += stride) ws.tile_mask[i] = 0u;
  if (zero_all && tid == 0) {
    ws.totals[2] = 0;   // centres handed to the CTA-per-centre backward
    ws.totals[4] = 0;   // next centre of the AEV forward
    ws.totals[5] = 0;   // next centre of the warp-per-centre backward
  }
  if (!rebuild) {
    // persistent lists: the grids and counts of the last build stay; only this
    // call's pointers are new, and the forces start again from zero
    if (tid < bp.n_sys) ws.sys[bp.sys_base + tid].in = bp.sys[tid];
    if (zero_all)
      for (int i = tid; i < n_in; i += stride) ws.f_pos[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  if (tid < bp.n_sys) {
    SysDev d;
    d.in = bp.sys[tid];
    d.n_ml = 0;
    d.atom_base = 0;
    d.cell_base = 0;
    for (int c = 0; c < 3; ++c) {
      d.nc[c] = 1;
      d.origin[c] = 0.f;
      d.inv_cell[c] = 0.f;
      d.bb_min[c] = 0xffffffffu;
      d.bb_max[c] = 0u;
    }
    ws.sys[bp.sys_base + tid] = d;
  }
  if (!zero_all) return;
  if (tid < kMaxSpecies) {
    ws.species_count[tid] = 0;
    ws.species_fill[tid] = 0;
  }
  if (tid < 4) ws.totals[tid] = 0;
  // the batch's cell grids hold at most 2 n + 27 cells per system (k_setup)
  const int cells = min(ws.cell_cap, 2 * n_in + 27 * ws.n_sys);
  for (int i = tid; i < cells; i += stride) ws.cell_count[i] = 0;
  for (int i = tid; i < n_in; i += stride) ws.f_pos[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void k_init(Ws ws, BatchParams bp, int zero_all, int n_in) {
  init_body(ws, bp, zero_all, n_in, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// one input atom of a chunk (all 32 lanes of a warp call it together)
__device__ __forceinline__ void prep_body(const Ws& ws, const BatchParams& bp, int t, int n_chunk,
                                          int S) {
  const unsigned lane = threadIdx.x & 31;
  const bool live = t < n_chunk;
  int k = 0, local = 0, gi = 0, s = -1, b = -1;
  bool ml = false;
  float x = 0.f, y = 0.f, z = 0.f;
  if (live) {
    k = find_sys(bp, t);
    const SysIn& si = bp.sys[k];
    local = t - (si.in_base - bp.sys[0].in_base);
    gi = si.in_base + local;
    b = bp.sys_base + k;
    ml = (si.mask == nullptr) || (si.mask[local] != 0);
    // every output force starts at zero (atoms outside the mask keep it)
    if (si.forces) {
      si.forces[3 * local + 0] = 0.f;
      si.forces[3 * local + 1] = 0.f;
      si.forces[3 * local + 2] = 0.f;
    }
    if (si.atom_e) si.atom_e[local] = 0.f;
    if (si.dLdR) {
      si.dLdR[3 * local + 0] = 0.f;
      si.dLdR[3 * local + 1] = 0.f;
      si.dLdR[3 * local + 2] = 0.f;
    }
    if (local == 0) {
      *si.energy = 0.0;
      if (si.virial)
        for (int c = 0; c < 9; ++c) si.virial[c] = 0.0;
    }
    if (ml) {
      s = si.species[local];
      x = si.coords[3 * local + 0];
      y = si.coords[3 * local + 1];
      z = si.coords[3 * local + 2];
      int bad = 0;
      if (s >= S) bad |= kStSpecies;
      if (!isfinite(x) || !isfinite(y) || !isfinite(z)) bad |= kStNonFinite;
      if (bad) {
        atomicOr(ws.status, bad);
        ml = false;  // excluded; the call reports the error
      }
    }
    ws.in_sys[gi] = ml ? b : -1;
  }
  if (!lists_rebuild(ws)) return;   // persistent lists: counts and boxes of the last build
  if (live && ws.in_pos) ws.in_pos[gi] = -1;
  // per-system ML atom counts and bounding boxes (warp-aggregated)
  const unsigned act = __ballot_sync(0xffffffffu, live && ml);
  if (live && ml) {
    const unsigned grp = __match_any_sync(act, b);
    const int leader = __ffs(grp) - 1;
    if ((int)lane == leader) atomicAdd(&ws.sys[b].n_ml, __popc(grp));
    if (!bp.sys[k].periodic) {
      const float v[3] = {x, y, z};
      for (int c = 0; c < 3; ++c) {
        const unsigned key = float_key(v[c]);
        const unsigned mn = __reduce_min_sync(grp, key);
        const unsigned mx = __reduce_max_sync(grp, key);
        if ((int)lane == leader) {
          atomicMin(&ws.sys[b].bb_min[c], mn);
          atomicMax(&ws.sys[b].bb_max[c], mx);
        }
      }
    }
    const unsigned sg = __match_any_sync(act, s);
    if ((int)lane == __ffs(sg) - 1) atomicAdd(&ws.species_count[s], __popc(sg));
  }
}

__global__ void k_prep(Ws ws, BatchParams bp, int n_chunk, int S) {
  prep_body(ws, bp, blockIdx.x * blockDim.x + threadIdx.x, n_chunk, S);
}

// block-wide exclusive scan helper (blockDim.x a multiple of 32, at most 1024)
__device__ int block_exclusive_scan(int v, int* total) {
  __shared__ int warp_sums[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) warp_sums[w] = incl;
  __syncthreads();
  if (w == 0) {
    int ws_ = lane < nw ? warp_sums[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, ws_, o);
      if (lane >= o) ws_ += u;
    }
    if (lane < nw) warp_sums[lane] = ws_;
  }
  __syncthreads();
  const int before = (w > 0 ? warp_sums[w - 1] : 0) + incl - v;
  *total = warp_sums[nw - 1];
  __syncthreads();
  return before;
}

__device__ __forceinline__ void setup_body(const Ws& ws, const AevConst& ac) {
  if (!lists_rebuild(ws)) return;
  const float rc = fmaxf(ac.rc_r, ac.rc_a) + ac.skin;
  int run_atoms = 0, run_cells = 0;
  for (int b0 = 0; b0 < ws.n_sys; b0 += blockDim.x) {
    const int b = b0 + threadIdx.x;
    int n_ml = 0, ncell = 0;
    SysDev d;
    if (b < ws.n_sys) {
      d = ws.sys[b];
      n_ml = d.n_ml;
      const long long cap = 2LL * d.in.n_in + 27;
      int nc[3];
      float len[3], org[3];
      for (int c = 0; c < 3; ++c) {
        if (d.in.periodic) {
          len[c] = d.in.box_hi[c];
          org[c] = 0.f;
        } else if (n_ml > 0) {
          const float lo = key_float(d.bb_min[c]), hi = key_float(d.bb_max[c]);
          len[c] = fmaxf(hi - lo, 1e-3f);
          org[c] = lo;
        } else {
          len[c] = 1.f;
          org[c] = 0.f;
        }
      }
      cell_grid(len, rc, cap, nc);
      for (int c = 0; c < 3; ++c) {
        d.nc[c] = nc[c];
        d.origin[c] = org[c];
        d.inv_cell[c] = nc[c] / len[c];
      }
      ncell = nc[0] * nc[1] * nc[2];
    }
    int tot_a, tot_c;
    const int ea = block_exclusive_scan(n_ml, &tot_a);
    const int ec = block_exclusive_scan(ncell, &tot_c);
    if (b < ws.n_sys) {
      d.atom_base = run_atoms + ea;
      d.cell_base = run_cells + ec;
      ws.sys[b] = d;
    }
    run_atoms += tot_a;
    run_cells += tot_c;
  }
  if (threadIdx.x == 0) {
    // more cells than the arena holds (impossible while the arena is sized for
    // 2 n + 27 cells per system, as every grid is): the call reports it, and the
    // batch becomes empty for every later kernel (no atoms, cells or AEV rows),
    // so that no kernel indexes past the cell arrays
    const bool over = run_cells > ws.cell_cap;
    if (over) atomicOr(ws.status, kStCells);
    ws.totals[0] = over ? 0 : run_atoms;
    ws.totals[1] = over ? 0 : run_cells;
    int acc = 0;
    for (int s = 0; s < ac.S; ++s) {
      ws.seg_start[s] = acc;
      if (!over) acc += (ws.species_count[s] + kRowTile - 1) / kRowTile * kRowTile;
    }
    for (int s = ac.S; s <= kMaxSpecies; ++s) ws.seg_start[s] = acc;
  }
}

// the cell grids of this batch fit the arena (k_setup clears the batch otherwise)
__device__ __forceinline__ bool cells_fit(const Ws& ws) {
  return (*(volatile const int*)ws.status & kStCells) == 0;
}

__global__ void k_setup(Ws ws, AevConst ac) { setup_body(ws, ac); }

// periodic systems: the coordinate wrapped into [0, L] (the value the cell index
// is taken from and the one stored for the kernels); else the coordinate itself
__device__ __forceinline__ float wrap_coord(float x, const SysDev& d, int c) {
  if (!d.in.periodic) return x;
  const float L = d.in.box_hi[c];
  return x - floorf(x / L) * L;   // exact for x already in [0, L)
}

__device__ __forceinline__ int cell_coord(float x, const SysDev& d, int c) {
  const float u = d.in.periodic ? wrap_coord(x, d, c) : x - d.origin[c];
  int k = (int)floorf(u * d.inv_cell[c]);
  return min(max(k, 0), d.nc[c] - 1);
}

// one input atom (all 32 lanes of a warp call it together)
__device__ __forceinline__ void bin_body(const Ws& ws, int gi, int n_in) {
  if (!cells_fit(ws)) return;   // uniform: the flag is set before this kernel (or phase)
  const unsigned lane = threadIdx.x & 31;
  int b = -1;
  if (gi < n_in) b = ws.in_sys[gi];
  const bool ml = b >= 0;
  const unsigned act = __ballot_sync(0xffffffffu, ml);
  if (!ml) return;
  const SysDev& d = ws.sys[b];
  const int local = gi - d.in.in_base;
  const float x = d.in.coords[3 * local + 0];
  const float y = d.in.coords[3 * local + 1];
  const float z = d.in.coords[3 * local + 2];
  const int s = d.in.species[local];
  const int cx = cell_coord(x, d, 0), cy = cell_coord(y, d, 1), cz = cell_coord(z, d, 2);
  const int gcell = d.cell_base + (cx * d.nc[1] + cy) * d.nc[2] + cz;
  if (!NNP_IN_BOUNDS(ws.status, kSiteBinCell, gcell, ws.cell_cap)) return;
  const int rank = atomicAdd(&ws.cell_count[gcell], 1);
  const unsigned sg = __match_any_sync(act, s);
  const int leader = __ffs(sg) - 1;
  int base = 0;
  if ((int)lane == leader) base = atomicAdd(&ws.species_fill[s], __popc(sg));
  base = __shfl_sync(sg, base, leader);
  const int slot = ws.seg_start[s] + base + __popc(sg & lanemask_lt());
  ws.in_cell[gi] = gcell;
  ws.in_rank[gi] = rank;
  ws.in_slot[gi] = slot;
}

__global__ void k_bin(Ws ws, int n_in) {
  if (!lists_rebuild(ws)) return;
  bin_body(ws, blockIdx.x * blockDim.x + threadIdx.x, n_in);
}

// single-block exclusive scan of the cell counts (1024 threads)
__device__ __forceinline__ void scan_body(const Ws& ws) {
  __shared__ int warp_sums[32];
  const int T = ws.totals[1];
  const int nt = blockDim.x;
  const int per = (T + nt - 1) / nt;
  const int beg = min(T, threadIdx.x * per), end = min(T, beg + per);
  int sum = 0;
  for (int i = beg; i < end; ++i) sum += ws.cell_count[i];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int incl = sum;
  for (int o = 1; o < 32; o <<= 1) {
    int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) warp_sums[w] = incl;
  __syncthreads();
  if (w == 0) {
    int v = warp_sums[lane];
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    warp_sums[lane] = v;
  }
  __syncthreads();
  int run = (w > 0 ? warp_sums[w - 1] : 0) + incl - sum;
  for (int i = beg; i < end; ++i) {
    ws.cell_start[i] = run;
    run += ws.cell_count[i];
  }
  if (threadIdx.x == nt - 1) ws.cell_start[T] = warp_sums[31];
}

__global__ void k_scan(Ws ws) {
  if (!lists_rebuild(ws)) return;
  scan_body(ws);
}

__device__ __forceinline__ void scatter_body(const Ws& ws, int gi, int n_in) {
  if (gi >= n_in) return;
  if (!lists_rebuild(ws)) {
    // persistent lists: new coordinates into the packed order of the last build
    const int pos = ws.in_pos[gi];
    if (pos < 0) return;
    const SysDev& d = ws.sys[ws.pos_sys[pos]];
    const int local = gi - d.in.in_base;
    ws.xyzq[pos] = make_float4(wrap_coord(d.in.coords[3 * local + 0], d, 0),
                               wrap_coord(d.in.coords[3 * local + 1], d, 1),
                               wrap_coord(d.in.coords[3 * local + 2], d, 2), ws.xyzq[pos].w);
    return;
  }
  const int b = ws.in_sys[gi];
  if (b < 0 || !cells_fit(ws)) return;
  const SysDev& d = ws.sys[b];
  const int local = gi - d.in.in_base;
  const int gcell = ws.in_cell[gi];
  const int pos = ws.cell_start[gcell] + ws.in_rank[gi];
  const int slot = ws.in_slot[gi];
  if (!NNP_IN_BOUNDS(ws.status, kSiteScatterPos, pos, n_in)) return;
  if (!NNP_IN_BOUNDS(ws.status, kSiteAevRow, slot, ws.row_cap)) return;
  ws.xyzq[pos] = make_float4(wrap_coord(d.in.coords[3 * local + 0], d, 0),
                             wrap_coord(d.in.coords[3 * local + 1], d, 1),
                             wrap_coord(d.in.coords[3 * local + 2], d, 2),
                             __int_as_float((int)d.in.species[local]));
  ws.pos_src[pos] = gi;
  ws.pos_slot[pos] = slot;
  if (ws.slot_pos) ws.slot_pos[slot] = pos;
  ws.pos_sys[pos] = b;
  ws.pos_cell[pos] = gcell - d.cell_base;
  if (ws.in_pos) {   // the reference the displacement check of later calls compares with
    ws.in_pos[gi] = pos;
    ws.ref[gi] = make_float4(d.in.coords[3 * local + 0], d.in.coords[3 * local + 1],
                             d.in.coords[3 * local + 2], 0.f);
  }
}

__global__ void k_scatter(Ws ws, int n_in) {
  scatter_body(ws, blockIdx.x * blockDim.x + threadIdx.x, n_in);
}

// The whole front end (init, prep, setup, bin, scan, scatter) of a one-chunk
// batch in a single CTA: one launch instead of six for small batches, with
// __syncthreads between the phases (their global writes are visible to the
// whole CTA after the barrier).
constexpr int kFrontThreads = 1024;
__global__ void __launch_bounds__(kFrontThreads) k_front(Ws ws, BatchParams bp, AevConst ac,
                                                          int n_in) {
  const int tid = threadIdx.x;
  init_body(ws, bp, 1, n_in, tid, kFrontThreads);
  __syncthreads();
  const int n_up = (n_in + 31) & ~31;   // whole warps, for the warp-collective parts
  for (int t = tid; t < n_up; t += kFrontThreads) prep_body(ws, bp, t, n_in, ac.S);
  __syncthreads();
  setup_body(ws, ac);
  __syncthreads();
  for (int t = tid; t < n_up; t += kFrontThreads) bin_body(ws, t, n_in);
  __syncthreads();
  scan_body(ws);
  __syncthreads();
  for (int t = tid; t < n_in; t += kFrontThreads) scatter_body(ws, t, n_in);
}

// Largest displacement of an atom of the last build's lists since that build
// (minimum image in periodic directions), as float bits into skin_state[0]
// (positive floats order like their bit patterns).
__global__ void k_skin_check(Ws ws, BatchParams bp, int n_chunk) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  float d2 = 0.f;
  if (t < n_chunk) {
    const int k = find_sys(bp, t);
    const SysIn& si = bp.sys[k];
    const int local = t - (si.in_base - bp.sys[0].in_base);
    const int gi = si.in_base + local;
    if (ws.in_pos[gi] >= 0) {
      const float4 r0 = ws.ref[gi];
      float d[3] = {si.coords[3 * local + 0] - r0.x, si.coords[3 * local + 1] - r0.y,
                    si.coords[3 * local + 2] - r0.z};
      if (si.periodic)
        for (int c = 0; c < 3; ++c) {
          const float n = rintf(d[c] / si.box_hi[c]);
          d[c] = fmaf(-n, si.box_lo[c], fmaf(-n, si.box_hi[c], d[c]));
        }
      d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (!(d2 == d2)) d2 = 3.0e38f;   // a non-finite coordinate forces a rebuild
    }
  }
  const int key = (int)__reduce_max_sync(0xffffffffu, __float_as_uint(sqrtf(d2)));
  if ((threadIdx.x & 31) == 0 && key > 0) atomicMax(ws.skin_state, key);
}

// Neighbour lists of centre p by one warp, candidates read from global memory
// and staged in st_j / st_t (kStageCap each), then species-sorted.  Used for
// home cells whose 27-cell neighbourhood does not fit the shared-memory stage
// of k_neighbors.
__device__ void centre_lists_global(const Ws& ws, const AevConst& ac, int p, int* st_j,
                                    uint8_t* st_t) {
  const unsigned lane = threadIdx.x & 31;
  __syncwarp();   // the stage may still be read by the warp's previous centre
  const float4 xi = ws.xyzq[p];
  const int b = ws.pos_sys[p];
  const SysDev& d = ws.sys[b];
  const int per = d.in.periodic;
  const int lc = ws.pos_cell[p];
  const int nc0 = d.nc[0], nc1 = d.nc[1], nc2 = d.nc[2];
  const int c2 = lc % nc2, c1 = (lc / nc2) % nc1, c0 = lc / (nc1 * nc2);
  const float rl = ac.rc_r + ac.skin, al = ac.rc_a + ac.skin;   // list cutoffs
  const float rr2 = rl * rl, ra2 = al * al;
  const float Lh0 = d.in.box_hi[0], Lh1 = d.in.box_hi[1], Lh2 = d.in.box_hi[2];
  const float Ll0 = d.in.box_lo[0], Ll1 = d.in.box_lo[1], Ll2 = d.in.box_lo[2];
  const float iL0 = per ? 1.f / Lh0 : 0.f, iL1 = per ? 1.f / Lh1 : 0.f, iL2 = per ? 1.f / Lh2 : 0.f;
  int cnt = 0;
  // candidate cell index lists per dimension (distinct cells only)
  int cl0[3], cl1[3], cl2[3], n0 = 0, n1 = 0, n2 = 0;
  {
    const int cc[3] = {c0, c1, c2};
    const int ncv[3] = {nc0, nc1, nc2};
    int* out[3] = {cl0, cl1, cl2};
    int* nout[3] = {&n0, &n1, &n2};
    for (int c = 0; c < 3; ++c) {
      int m = 0;
      if (ncv[c] >= 3 || !per) {
        for (int o = -1; o <= 1; ++o) {
          int k = cc[c] + o;
          if (per) k = (k + ncv[c]) % ncv[c];
          else if (k < 0 || k >= ncv[c]) continue;
          out[c][m++] = k;
        }
      } else {
        for (int k = 0; k < ncv[c]; ++k) out[c][m++] = k;
      }
      *nout[c] = m;
    }
  }
  // z-neighbour cells that are consecutive in the cell order form one range of
  // the cell-sorted atoms: sort the (at most 3) z indices and merge runs
  int zs[3];
  for (int a2 = 0; a2 < n2; ++a2) zs[a2] = cl2[a2];
  for (int a = 0; a < n2; ++a)
    for (int b = a + 1; b < n2; ++b)
      if (zs[b] < zs[a]) { const int t = zs[a]; zs[a] = zs[b]; zs[b] = t; }
  int zr_beg[3], zr_end[3], nzr = 0;
  for (int a2 = 0; a2 < n2; ++a2) {
    if (nzr > 0 && zs[a2] == zr_end[nzr - 1]) {
      zr_end[nzr - 1] = zs[a2] + 1;
    } else {
      zr_beg[nzr] = zs[a2];
      zr_end[nzr] = zs[a2] + 1;
      ++nzr;
    }
  }
  for (int a0 = 0; a0 < n0; ++a0)
    for (int a1 = 0; a1 < n1; ++a1)
      for (int zr = 0; zr < nzr; ++zr) {
        const int row = d.cell_base + (cl0[a0] * nc1 + cl1[a1]) * nc2;
        const int beg = ws.cell_start[row + zr_beg[zr]], end = ws.cell_start[row + zr_end[zr]];
        for (int j0 = beg; j0 < end; j0 += 32) {
          const int j = j0 + lane;
          bool keep = false, ang = false;
          int sj = 0;
          if (j < end && j != p) {
            const float4 xj = ws.xyzq[j];
            float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
            if (per) {
              float n;
              n = rintf(dx * iL0); dx = fmaf(-n, Lh0, dx); dx = fmaf(-n, Ll0, dx);
              n = rintf(dy * iL1); dy = fmaf(-n, Lh1, dy); dy = fmaf(-n, Ll1, dy);
              n = rintf(dz * iL2); dz = fmaf(-n, Lh2, dz); dz = fmaf(-n, Ll2, dz);
            }
            const float r2 = dx * dx + dy * dy + dz * dz;
            keep = (r2 <= rr2) && (r2 > 1e-12f);
            ang = keep && (r2 <= ra2);
            sj = __float_as_int(xj.w);
          }
          const unsigned bal = __ballot_sync(0xffffffffu, keep);
          if (keep) {
            const int at = cnt + __popc(bal & lanemask_lt());
            if (at < kStageCap) {
              st_j[at] = j;
              st_t[at] = (uint8_t)(sj | (ang ? 0x80 : 0));
            }
          }
          cnt += __popc(bal);
        }
      }
  __syncwarp();
  const int nst = min(cnt, kStageCap);
  // species-sorted radial and angular lists
  int wr_r = 0, wr_a = 0;
  uint16_t* hdr = ws.nb_cnt + (size_t)p * 16;
  int* out_r = ws.nb_r + (size_t)p * ws.cap_r;
  int* out_a = ws.nb_a + (size_t)p * ws.cap_a;
  for (int s = 0; s < ac.S; ++s) {
    int cr = 0, ca = 0;
    for (int t0 = 0; t0 < nst; t0 += 32) {
      const int t = t0 + lane;
      bool mr = false, ma = false;
      int j = 0;
      if (t < nst) {
        const int tt = st_t[t];
        j = st_j[t];
        mr = (tt & 0x7f) == s;
        ma = mr && (tt & 0x80);
      }
      const unsigned br = __ballot_sync(0xffffffffu, mr);
      const unsigned ba = __ballot_sync(0xffffffffu, ma);
      if (mr) {
        const int at = wr_r + cr + __popc(br & lanemask_lt());
        if (at < ws.cap_r && NNP_IN_BOUNDS(ws.status, kSiteNbCandidate, j, ws.totals[0])) out_r[at] = j;
      }
      if (ma) {
        const int at = wr_a + ca + __popc(ba & lanemask_lt());
        if (at < ws.cap_a && NNP_IN_BOUNDS(ws.status, kSiteNbCandidate, j, ws.totals[0])) out_a[at] = j;
      }
      cr += __popc(br);
      ca += __popc(ba);
    }
    // clamp the per-species counts so that the lists stay inside their capacity
    const int keep_r = max(0, min(cr, ws.cap_r - wr_r));
    const int keep_a = max(0, min(ca, ws.cap_a - wr_a));
    if (lane == 0) {
      hdr[s] = (uint16_t)keep_r;
      hdr[8 + s] = (uint16_t)keep_a;
    }
    wr_r += cr;
    wr_a += ca;
  }
  if (lane == 0) {
    for (int s = ac.S; s < 8; ++s) { hdr[s] = 0; hdr[8 + s] = 0; }
    if (cnt > ws.cap_r || wr_a > ws.cap_a || cnt > kStageCap) {
      atomicOr(ws.status, kStCapacity);
      atomicMax(ws.status + 1, cnt);
      atomicMax(ws.status + 2, wr_a);
    }
  }
}


// Species-sorted radial (R <= rc_r) and angular (R <= rc_a) lists of centre p
// from the candidates cand[t] / cand_j[t], t in [sp_start[s], sp_start[s+1])
// for species s (coordinates already shifted to the centre's periodic image;
// dimensions flagged in min_img take the minimum image per pair instead).  With
// idx, position t of the scan is candidate idx[t] (a subset of the candidates in
// their order, sp_start counting positions of idx).
__device__ __forceinline__ void centre_lists_staged(const Ws& ws, const AevConst& ac, int p,
                                                    const float4* cand, const int* cand_j,
                                                    const int* sp_start, const int* min_img,
                                                    const SysDev& d,
                                                    const uint16_t* idx = nullptr) {
  const unsigned lane = threadIdx.x & 31;
  const float4 xi = ws.xyzq[p];
  const float rl = ac.rc_r + ac.skin, al = ac.rc_a + ac.skin;   // list cutoffs
  const float rr2 = rl * rl, ra2 = al * al;
  const bool any_mi = min_img[0] | min_img[1] | min_img[2];
  uint16_t* hdr = ws.nb_cnt + (size_t)p * 16;
  int* out_r = ws.nb_r + (size_t)p * ws.cap_r;
  int* out_a = ws.nb_a + (size_t)p * ws.cap_a;
  int wr_r = 0, wr_a = 0;
  // candidate t of the staged list: within the radial / angular list cutoff?
  auto test = [&](int t, int end, int& j, bool& keep, bool& ang) {
    keep = ang = false;
    j = 0;
    if (t < end) {
      const int c = idx ? (int)idx[t] : t;
      const float4 xj = cand[c];
      j = cand_j[c];
      float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
      if (any_mi) {
        float n;
        if (min_img[0]) { n = rintf(dx / d.in.box_hi[0]); dx = fmaf(-n, d.in.box_hi[0], dx); dx = fmaf(-n, d.in.box_lo[0], dx); }
        if (min_img[1]) { n = rintf(dy / d.in.box_hi[1]); dy = fmaf(-n, d.in.box_hi[1], dy); dy = fmaf(-n, d.in.box_lo[1], dy); }
        if (min_img[2]) { n = rintf(dz / d.in.box_hi[2]); dz = fmaf(-n, d.in.box_hi[2], dz); dz = fmaf(-n, d.in.box_lo[2], dz); }
      }
      const float r2 = dx * dx + dy * dy + dz * dz;
      keep = (r2 <= rr2) && (r2 > 1e-12f) && (j != p);
      ang = keep && (r2 <= ra2);
    }
  };
  for (int s = 0; s < ac.S; ++s) {
    int cr = 0, ca = 0;
    const int end = sp_start[s + 1];
    // two 32-candidate chunks per pass (independent loads and tests), appended
    // in candidate order
    for (int t0 = sp_start[s]; t0 < end; t0 += 64) {
      int j0, j1;
      bool k0, a0, k1, a1;
      test(t0 + (int)lane, end, j0, k0, a0);
      test(t0 + 32 + (int)lane, end, j1, k1, a1);
      const unsigned br0 = __ballot_sync(0xffffffffu, k0), ba0 = __ballot_sync(0xffffffffu, a0);
      const unsigned br1 = __ballot_sync(0xffffffffu, k1), ba1 = __ballot_sync(0xffffffffu, a1);
      const unsigned lt = lanemask_lt();
      if (k0) {
        const int at = wr_r + cr + __popc(br0 & lt);
        if (at < ws.cap_r && NNP_IN_BOUNDS(ws.status, kSiteNbCandidate, j0, ws.totals[0])) out_r[at] = j0;
      }
      if (a0) {
        const int at = wr_a + ca + __popc(ba0 & lt);
        if (at < ws.cap_a && NNP_IN_BOUNDS(ws.status, kSiteNbCandidate, j0, ws.totals[0])) out_a[at] = j0;
      }
      cr += __popc(br0);
      ca += __popc(ba0);
      if (k1) {
        const int at = wr_r + cr + __popc(br1 & lt);
        if (at < ws.cap_r && NNP_IN_BOUNDS(ws.status, kSiteNbCandidate, j1, ws.totals[0])) out_r[at] = j1;
      }
      if (a1) {
        const int at = wr_a + ca + __popc(ba1 & lt);
        if (at < ws.cap_a && NNP_IN_BOUNDS(ws.status, kSiteNbCandidate, j1, ws.totals[0])) out_a[at] = j1;
      }
      cr += __popc(br1);
      ca += __popc(ba1);
    }
    const int keep_r = max(0, min(cr, ws.cap_r - wr_r));
    const int keep_a = max(0, min(ca, ws.cap_a - wr_a));
    if (lane == 0) {
      hdr[s] = (uint16_t)keep_r;
      hdr[8 + s] = (uint16_t)keep_a;
    }
    wr_r += cr;
    wr_a += ca;
  }
  if (lane == 0) {
    for (int s = ac.S; s < 8; ++s) { hdr[s] = 0; hdr[8 + s] = 0; }
    if (wr_r > ws.cap_r || wr_a > ws.cap_a || wr_r > kStageCap) {
      atomicOr(ws.status, kStCapacity);
      atomicMax(ws.status + 1, wr_r);
      atomicMax(ws.status + 2, wr_a);
    }
  }
}

constexpr int kNbThreads = 256;   // 8 warps
constexpr int kCandCap = 2048;    // staged candidates of one home cell
constexpr int kOctCap = 512;      // candidates of one octant list
constexpr int kOctMin = 256;      // octant lists only for more candidates than this

// octant of a point of the home cell about the cell's centre mid
__device__ __forceinline__ int octant_of(const float4& x, const float* mid) {
  return (x.x >= mid[0] ? 1 : 0) | (x.y >= mid[1] ? 2 : 0) | (x.z >= mid[2] ? 4 : 0);
}

// One CTA per home cell (grid-stride over the cells of the batch).  The atoms of
// the 27 neighbour cells are staged once in shared memory, shifted to the home
// cell's periodic image and stably sorted by species; then one warp per centre
// of the home cell scans them species by species and appends the accepted
// neighbours to its lists, which come out species-sorted without a sort pass.
__global__ void __launch_bounds__(kNbThreads) k_neighbors(Ws ws, AevConst ac) {
  __shared__ float4 cand[kCandCap];
  __shared__ int cand_j[kCandCap];
  __shared__ uint16_t chunk_cnt[kCandCap / 32][kMaxSpecies];
  __shared__ int r_beg[27], r_off[28];
  __shared__ float r_shift[27][3];
  __shared__ int sp_start[kMaxSpecies + 1];
  __shared__ int min_img[3];
  // octant lists: the candidates (positions in cand, in order) within the list
  // cutoff of the bounding box of the home cell's atoms in each octant
  __shared__ uint16_t oct_idx[8][kOctCap];
  __shared__ int oct_sp[8][kMaxSpecies + 1];
  __shared__ int oct_n[8];
  __shared__ unsigned oct_key[8][6];   // box as order-preserving keys: min x y z, max x y z
  __shared__ float oct_mid[3];
  const int tid = threadIdx.x, w = tid >> 5;
  const unsigned lane = tid & 31;
  if (!lists_rebuild(ws)) return;
  const int n_cells = ws.totals[1];
  for (int gc = blockIdx.x; gc < n_cells; gc += gridDim.x) {
    const int cbeg = ws.cell_start[gc], cend = ws.cell_start[gc + 1];
    if (cbeg == cend) continue;   // uniform across the CTA
    const int b = ws.pos_sys[cbeg];
    const SysDev& d = ws.sys[b];
    const int per = d.in.periodic;
    const int nc[3] = {d.nc[0], d.nc[1], d.nc[2]};
    const int lc = gc - d.cell_base;
    const int cc[3] = {lc / (nc[1] * nc[2]), (lc / nc[2]) % nc[1], lc % nc[2]};
    // ---- the 27 (or fewer) neighbour cells: thread t < 27 takes offset (t/9, t/3%3, t%3)
    if (w == 0) {
      int cnt = 0, beg = 0;
      float sh[3] = {0.f, 0.f, 0.f};
      if (lane < 27) {
        const int o[3] = {(int)lane / 9, ((int)lane / 3) % 3, (int)lane % 3};
        bool ok = true;
        int k[3];
        for (int c = 0; c < 3; ++c) {
          if (per && nc[c] < 3) {
            // every cell of this dimension once, minimum image per pair
            k[c] = o[c];
            ok &= o[c] < nc[c];
          } else {
            k[c] = cc[c] + o[c] - 1;
            if (per) {
              if (k[c] < 0) { k[c] += nc[c]; sh[c] = -d.in.box_hi[c]; }
              else if (k[c] >= nc[c]) { k[c] -= nc[c]; sh[c] = d.in.box_hi[c]; }
            } else {
              ok &= (k[c] >= 0 && k[c] < nc[c]);
            }
          }
        }
        if (ok) {
          const int g = d.cell_base + (k[0] * nc[1] + k[1]) * nc[2] + k[2];
          beg = ws.cell_start[g];
          cnt = ws.cell_start[g + 1] - beg;
        }
        r_beg[lane] = beg;
        r_shift[lane][0] = sh[0]; r_shift[lane][1] = sh[1]; r_shift[lane][2] = sh[2];
      }
      int incl = cnt;
      for (int o2 = 1; o2 < 32; o2 <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o2);
        if ((int)lane >= o2) incl += u;
      }
      if (lane < 27) r_off[lane] = incl - cnt;
      if (lane == 26) r_off[27] = incl;
      if (lane < 3) min_img[lane] = (per && nc[lane] < 3) ? 1 : 0;
    }
    __syncthreads();
    const int total = r_off[27];
    if (total > kCandCap) {
      // too many candidates to stage: per-centre search from global memory,
      // with the candidate arrays as the warps' staging space
      int* stj = reinterpret_cast<int*>(cand) + w * kStageCap;
      uint8_t* stt = reinterpret_cast<uint8_t*>(reinterpret_cast<int*>(cand) + 8 * kStageCap) + w * kStageCap;
      for (int p = cbeg + w; p < cend; p += kNbThreads / 32) centre_lists_global(ws, ac, p, stj, stt);
      __syncthreads();
      continue;
    }
    const int n_chunks = (total + 31) >> 5;
    // ---- stable species sort of the candidates: counts per 32-chunk, offsets, placement
    for (int pass = 0; pass < 2; ++pass) {
      for (int ch = w; ch < n_chunks; ch += kNbThreads / 32) {
        const int q = ch * 32 + (int)lane;
        const bool valid = q < total;
        int r = 0;
        if (valid) {
          int lo = 0, hi = 26;   // last range with r_off <= q
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (r_off[mid] <= q) lo = mid; else hi = mid - 1;
          }
          r = lo;
        }
        const int j = valid ? r_beg[r] + q - r_off[r] : 0;
        const float4 xj = valid ? ws.xyzq[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int sp = valid ? __float_as_int(xj.w) : -1;
        if (pass == 0) {
          for (int s = 0; s < ac.S; ++s) {
            const unsigned bal = __ballot_sync(0xffffffffu, sp == s);
            if (lane == 0) chunk_cnt[ch][s] = (uint16_t)__popc(bal);
          }
        } else {
          const unsigned same = __match_any_sync(0xffffffffu, sp);
          if (valid) {
            const int pos = sp_start[sp] + chunk_cnt[ch][sp] + __popc(same & lanemask_lt());
            cand[pos] = make_float4(xj.x + r_shift[r][0], xj.y + r_shift[r][1], xj.z + r_shift[r][2], xj.w);
            cand_j[pos] = j;
          }
        }
      }
      __syncthreads();
      if (pass == 0) {
        if (tid < ac.S) {   // thread s: exclusive offsets of species s over the chunks
          int run = 0;
          for (int ch = 0; ch < n_chunks; ++ch) {
            const int v = chunk_cnt[ch][tid];
            chunk_cnt[ch][tid] = (uint16_t)run;
            run += v;
          }
          sp_start[tid + 1] = run;   // count for now
        }
        __syncthreads();
        if (tid == 0) {
          sp_start[0] = 0;
          for (int s = 0; s < ac.S; ++s) sp_start[s + 1] += sp_start[s];
        }
        __syncthreads();
      }
    }
    // ---- octant lists (when no dimension takes the minimum image per pair):
    // warp o keeps, species by species and in candidate order, the candidates
    // within the list cutoff of the bounding box of the home cell's atoms in
    // octant o; a centre then scans only its octant's list (the same neighbours
    // in the same order, a superset of them being tested).  A list longer than
    // kOctCap is not used; neighbourhoods of at most kOctMin candidates (small
    // molecules) are scanned whole, which costs less than building the lists.
    const bool use_oct = !(min_img[0] | min_img[1] | min_img[2]) && total > kOctMin;
    if (use_oct) {
      if (tid < 48) oct_key[tid / 6][tid % 6] = (tid % 6) < 3 ? 0xffffffffu : 0u;
      if (tid < 3) oct_mid[tid] = d.origin[tid] + ((float)cc[tid] + 0.5f) / d.inv_cell[tid];
      __syncthreads();
      for (int p = cbeg + tid; p < cend; p += kNbThreads) {
        const float4 x = ws.xyzq[p];
        const int o = octant_of(x, oct_mid);
        atomicMin(&oct_key[o][0], float_key(x.x));
        atomicMin(&oct_key[o][1], float_key(x.y));
        atomicMin(&oct_key[o][2], float_key(x.z));
        atomicMax(&oct_key[o][3], float_key(x.x));
        atomicMax(&oct_key[o][4], float_key(x.y));
        atomicMax(&oct_key[o][5], float_key(x.z));
      }
      __syncthreads();
      {
        const int o = w;
        int cnt = 0;
        if (oct_key[o][0] <= oct_key[o][3]) {   // the octant holds atoms
          const float lo[3] = {key_float(oct_key[o][0]), key_float(oct_key[o][1]), key_float(oct_key[o][2])};
          const float hi[3] = {key_float(oct_key[o][3]), key_float(oct_key[o][4]), key_float(oct_key[o][5])};
          // the centres' own test decides; this one only has to keep every
          // candidate it could accept, so its cutoff has a margin for rounding
          const float rl = ac.rc_r + ac.skin;
          const float rl2 = rl * rl * (1.f + 1e-5f) + 1e-6f;
          for (int s = 0; s < ac.S; ++s) {
            if (lane == 0) oct_sp[o][s] = cnt;
            const int end = sp_start[s + 1];
            for (int t0 = sp_start[s]; t0 < end; t0 += 32) {
              const int t = t0 + (int)lane;
              bool in = false;
              if (t < end) {
                const float4 c = cand[t];
                const float ex = fmaxf(fmaxf(lo[0] - c.x, c.x - hi[0]), 0.f);
                const float ey = fmaxf(fmaxf(lo[1] - c.y, c.y - hi[1]), 0.f);
                const float ez = fmaxf(fmaxf(lo[2] - c.z, c.z - hi[2]), 0.f);
                in = ex * ex + ey * ey + ez * ez <= rl2;
              }
              const unsigned bal = __ballot_sync(0xffffffffu, in);
              if (in) {
                const int at = cnt + __popc(bal & lanemask_lt());
                if (at < kOctCap) oct_idx[o][at] = (uint16_t)t;
              }
              cnt += __popc(bal);
            }
          }
          if (lane == 0) oct_sp[o][ac.S] = cnt;
        }
        if (lane == 0) oct_n[o] = cnt;
      }
      __syncthreads();
    }
    // ---- one warp per centre of the home cell
    for (int p = cbeg + w; p < cend; p += kNbThreads / 32) {
      if (use_oct) {
        const int o = octant_of(ws.xyzq[p], oct_mid);
        if (oct_n[o] <= kOctCap) {
          centre_lists_staged(ws, ac, p, cand, cand_j, oct_sp[o], min_img, d, oct_idx[o]);
          continue;
        }
      }
      centre_lists_staged(ws, ac, p, cand, cand_j, sp_start, min_img, d);
    }
    __syncthreads();   // the stage is rebuilt for the next home cell
  }
}

// Lists at the cutoffs from the persistent lists at the cutoffs + skin, one warp
// per centre: the entries of each species block of the longer radial list whose
// current distance is within rc_r (radial) or rc_a (angular), in their order.
__global__ void __launch_bounds__(256) k_list_refresh(Ws ws, AevConst ac) {
  const int p = blockIdx.x * 8 + (threadIdx.x >> 5);
  const unsigned lane = threadIdx.x & 31;
  if (p >= ws.totals[0]) return;
  const float4 xi = ws.xyzq[p];
  const SysDev& d = ws.sys[ws.pos_sys[p]];
  const int per = d.in.periodic;
  const float rr2 = ac.rc_r * ac.rc_r, ra2 = ac.rc_a * ac.rc_a;
  const uint16_t* hm = ws.nbs_cnt + (size_t)p * 16;
  const int* lm = ws.nbs_r + (size_t)p * ws.cap_r;
  uint16_t* hdr = ws.nb_cnt + (size_t)p * 16;
  int* out_r = ws.nb_r + (size_t)p * ws.cap_r;
  int* out_a = ws.nb_a + (size_t)p * ws.cap_a;
  int off = 0, wr_r = 0, wr_a = 0;
  for (int s = 0; s < ac.S; ++s) {
    const int end = off + hm[s];
    int cr = 0, ca = 0;
    for (int t0 = off; t0 < end; t0 += 32) {
      const int t = t0 + (int)lane;
      bool keep = false, ang = false;
      int j = 0;
      if (t < end) {
        j = lm[t];
        const float4 xj = ws.xyzq[j];
        float dv[3] = {xj.x - xi.x, xj.y - xi.y, xj.z - xi.z};
        if (per)
          for (int c = 0; c < 3; ++c) {
            const float n = rintf(dv[c] / d.in.box_hi[c]);
            dv[c] = fmaf(-n, d.in.box_lo[c], fmaf(-n, d.in.box_hi[c], dv[c]));
          }
        const float r2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
        keep = r2 <= rr2 && r2 > 1e-12f;
        ang = keep && r2 <= ra2;
      }
      const unsigned br = __ballot_sync(0xffffffffu, keep);
      const unsigned ba = __ballot_sync(0xffffffffu, ang);
      if (keep) {
        const int at = wr_r + cr + __popc(br & lanemask_lt());
        if (at < ws.cap_r && NNP_IN_BOUNDS(ws.status, kSiteNbCandidate, j, ws.totals[0])) out_r[at] = j;
      }
      if (ang) {
        const int at = wr_a + ca + __popc(ba & lanemask_lt());
        if (at < ws.cap_a && NNP_IN_BOUNDS(ws.status, kSiteNbCandidate, j, ws.totals[0])) out_a[at] = j;
      }
      cr += __popc(br);
      ca += __popc(ba);
    }
    // counts clamped so that the lists stay inside their capacity
    if (lane == 0) {
      hdr[s] = (uint16_t)max(0, min(cr, ws.cap_r - wr_r));
      hdr[8 + s] = (uint16_t)max(0, min(ca, ws.cap_a - wr_a));
    }
    wr_r += cr;
    wr_a += ca;
    off = end;
  }
  if (lane == 0) {
    for (int s = ac.S; s < 8; ++s) { hdr[s] = 0; hdr[8 + s] = 0; }
    if (wr_r > ws.cap_r || wr_a > ws.cap_a) {   // the call reports it; the retry grows the lists
      atomicOr(ws.status, kStCapacity);
      atomicMax(ws.status + 1, wr_r);
      atomicMax(ws.status + 2, wr_a);
    }
  }
}

}  // namespace

void launch_init_chunk(const Ws& ws, const BatchParams& bp, cudaStream_t st) {
  // the first chunk of a batch also zeroes the shared counters
  const int zero_all = (bp.sys_base == 0);
  const int cells = min(ws.cell_cap, 2 * ws.n_in + 27 * ws.n_sys);
  const int work = zero_all ? max(cells, max(ws.n_in, bp.n_sys)) : bp.n_sys;
  int blocks = (work + 255) / 256;
  blocks = max(1, min(blocks, 1184));
  k_init<<<blocks, 256, 0, st>>>(ws, bp, zero_all, ws.n_in);
}

void launch_prep_atoms(const Ws& ws, const BatchParams& bp, int n_in_chunk, int S,
                       cudaStream_t st) {
  if (n_in_chunk <= 0) return;
  k_prep<<<(n_in_chunk + 255) / 256, 256, 0, st>>>(ws, bp, n_in_chunk, S);
}

void launch_setup(const Ws& ws, const AevConst& ac, cudaStream_t st) {
  k_setup<<<1, 256, 0, st>>>(ws, ac);
}

void launch_bin(const Ws& ws, int n_in, cudaStream_t st) {
  if (n_in <= 0) return;
  k_bin<<<(n_in + 255) / 256, 256, 0, st>>>(ws, n_in);
}

void launch_scan(const Ws& ws, cudaStream_t st) { k_scan<<<1, 1024, 0, st>>>(ws); }

void launch_scatter(const Ws& ws, int n_in, cudaStream_t st) {
  if (n_in <= 0) return;
  k_scatter<<<(n_in + 255) / 256, 256, 0, st>>>(ws, n_in);
}

void launch_front(const Ws& ws, const BatchParams& bp, const AevConst& ac, int n_in,
                  cudaStream_t st) {
  k_front<<<1, kFrontThreads, 0, st>>>(ws, bp, ac, n_in);
}

void launch_skin_check(const Ws& ws, const BatchParams& bp, int n_in_chunk, cudaStream_t st) {
  if (n_in_chunk <= 0 || !ws.skin_state) return;
  k_skin_check<<<(n_in_chunk + 255) / 256, 256, 0, st>>>(ws, bp, n_in_chunk);
}

void launch_neighbors(const Ws& ws, int n_in, const AevConst& ac, cudaStream_t st) {
  if (n_in <= 0) return;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::max(1, std::min(ws.cell_cap, 4 * std::max(sms, 1)));
  if (ws.skin_state && ac.skin > 0.f) {
    // persistent lists: the search (when it runs) fills the lists at the cutoffs
    // + skin; every call then derives the lists at the cutoffs from them
    Ws wm = ws;
    wm.nb_cnt = ws.nbs_cnt;
    wm.nb_r = ws.nbs_r;
    wm.nb_a = ws.nbs_a;
    k_neighbors<<<grid, kNbThreads, 0, st>>>(wm, ac);
    k_list_refresh<<<(n_in + 7) / 8, 256, 0, st>>>(ws, ac);
  } else {
    k_neighbors<<<grid, kNbThreads, 0, st>>>(ws, ac);
  }
}

// ---------------------------------------------------------------- deterministic mode
namespace {

// one thread per cell: its packed atoms in input order (insertion sort by input
// index; a cell holds a few atoms), which the binning's atomic counter had
// placed in arrival order
__global__ void k_det_cell_sort(Ws ws) {
  if (!lists_rebuild(ws)) return;
  const int T = ws.totals[1];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < T; c += gridDim.x * blockDim.x) {
    const int b = ws.cell_start[c], e = ws.cell_start[c + 1];
    for (int i = b + 1; i < e; ++i) {
      const float4 x = ws.xyzq[i];
      const int src = ws.pos_src[i], sys = ws.pos_sys[i], cell = ws.pos_cell[i];
      int k = i - 1;
      while (k >= b && ws.pos_src[k] > src) {
        ws.xyzq[k + 1] = ws.xyzq[k];
        ws.pos_src[k + 1] = ws.pos_src[k];
        ws.pos_sys[k + 1] = ws.pos_sys[k];
        ws.pos_cell[k + 1] = ws.pos_cell[k];
        --k;
      }
      ws.xyzq[k + 1] = x;
      ws.pos_src[k + 1] = src;
      ws.pos_sys[k + 1] = sys;
      ws.pos_cell[k + 1] = cell;
    }
    if (ws.in_pos)
      for (int i = b; i < e; ++i) ws.in_pos[ws.pos_src[i]] = i;
  }
}

// one CTA: the AEV row of every packed atom, species segment by segment in
// packed order (the binning's atomic counter had assigned them in arrival order)
__global__ void __launch_bounds__(1024) k_det_slots(Ws ws, int S) {
  if (!lists_rebuild(ws)) return;
  __shared__ int next[kMaxSpecies];
  __shared__ int wcount[32][kMaxSpecies];
  const int n = ws.totals[0];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid < kMaxSpecies) next[tid] = tid < S ? ws.seg_start[tid] : 0;
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += 1024) {
    const int p = c0 + tid;
    const int s = p < n ? __float_as_int(ws.xyzq[p].w) : -1;
    int rank = 0;
    for (int q = 0; q < S; ++q) {
      const unsigned m = __ballot_sync(0xffffffffu, s == q);
      if (s == q) rank = __popc(m & lanemask_lt());
      if (lane == 0) wcount[w][q] = __popc(m);
    }
    __syncthreads();
    if (s >= 0 && s < S) {
      for (int k = 0; k < w; ++k) rank += wcount[k][s];
      const int slot = next[s] + rank;
      if (NNP_IN_BOUNDS(ws.status, kSiteAevRow, slot, ws.row_cap)) {
        ws.pos_slot[p] = slot;
        ws.in_slot[ws.pos_src[p]] = slot;
        if (ws.slot_pos) ws.slot_pos[slot] = p;
      }
    }
    __syncthreads();
    if (tid < S) {
      int tot = 0;
      for (int k = 0; k < 32; ++k) tot += wcount[k][tid];
      next[tid] += tot;
    }
    __syncthreads();
  }
}

}  // namespace

void launch_det_order(const Ws& ws, int S, cudaStream_t st) {
  if (!ws.fr_det) return;
  k_det_cell_sort<<<std::max(1, std::min((ws.cell_cap + 255) / 256, 1024)), 256, 0, st>>>(ws);
  k_det_slots<<<1, 1024, 0, st>>>(ws, S);
}

}  // namespace nnp
