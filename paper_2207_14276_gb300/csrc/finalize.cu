// Per-atom energies, the FP64 per-system energy reduction (paper Eq. 2) and the
// scatter of packed forces back to the caller's atom order; plus diagnostic
// gathers used by the parity tests.
#include "nnp_internal.cuh"

namespace nnp {

namespace {

__global__ void k_finalize(Ws ws, const float* e_row, int E, int e_row_net,
                           const double* ebias) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0 && ws.skin_state && lists_rebuild(ws)) {
    // the lists built in this call serve later calls unless they overflowed
    ws.skin_state[2] += 1;
    ws.skin_state[3] = (ws.status[0] & (kStCapacity | kStCells)) ? 0 : 1;
  }
  const unsigned lane = threadIdx.x & 31;
  const int total = ws.totals[0];
  const bool live = p < total;
  int b = -1;
  double Ei = 0.0;
  if (live) {
    b = ws.pos_sys[p];
    int slot = ws.pos_slot[p];
    if (!NNP_IN_BOUNDS(ws.status, kSiteFinalize, slot, ws.row_cap)) slot = 0;
    const int s = __float_as_int(ws.xyzq[p].w);
    float acc = 0.f;
    for (int e = 0; e < E; ++e) acc += e_row[(size_t)e * e_row_net + slot];
    Ei = (double)acc / (double)E + ebias[s];
    ws.atom_e[slot] = (float)Ei;
    const SysDev& d = ws.sys[b];
    const int local = ws.pos_src[p] - d.in.in_base;
    if (d.in.forces) {
      const float4 f = ws.f_pos[p];
      float* F = d.in.forces + 3 * (size_t)local;
      F[0] = f.x;
      F[1] = f.y;
      F[2] = f.z;
    }
    if (d.in.atom_e) d.in.atom_e[local] = (float)Ei;
  }
  // segmented FP64 reduction over the systems present in this warp
  unsigned todo = __ballot_sync(0xffffffffu, live);
  while (todo) {
    const int leader = __ffs(todo) - 1;
    const int key = __shfl_sync(0xffffffffu, b, leader);
    const bool mine = live && b == key;
    double v = mine ? Ei : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((int)lane == leader) atomicAdd(ws.sys[key].in.energy, v);
    todo &= ~__ballot_sync(0xffffffffu, mine);
  }
}

// out[src_atom][f] = rows[slot][col[f]] for f < D (rows of the batch's input
// atoms; col: the AEV column of feature f of the paper's order); rows: FP32, or
// (rows_h != null) BF16 bit patterns widened to FP32, plus the low BF16 parts
// rows_l of the split path if given
__global__ void k_gather_rows(Ws ws, const float* rows, const uint16_t* rows_h,
                              const uint16_t* rows_l, int ld, int D, const int16_t* col,
                              float* out, int by_tile) {
  const int p = blockIdx.x;
  if (p >= ws.totals[0]) return;
  const int slot = ws.pos_slot[p];
  const int gi = ws.pos_src[p];
  // sparse rows: 64-column slices outside the row's (AEV: zero) or the tile's
  // (dE/dG: not computed) mask read as 0
  const uint32_t m = !ws.row_mask ? ~0u : by_tile ? ws.tile_mask[slot >> 7] : ws.row_mask[slot];
  for (int f = threadIdx.x; f < D; f += blockDim.x) {
    const int c = col[f];
    const size_t i = (size_t)slot * ld + c;
    float v;
    if (!((m >> (c >> 6)) & 1u)) { out[(size_t)gi * D + f] = 0.f; continue; }
    if (rows_h) {
      v = __uint_as_float((unsigned)rows_h[i] << 16);
      if (rows_l) v += __uint_as_float((unsigned)rows_l[i] << 16);
    } else {
      v = rows[i];
    }
    out[(size_t)gi * D + f] = v;
  }
}

// out[src_atom][t] = input index of neighbour t (species-sorted), -1 past the count
__global__ void k_gather_nbrs(Ws ws, int angular, int cap_out, int* out) {
  const int p = blockIdx.x;
  if (p >= ws.totals[0]) return;
  const uint16_t* hdr = ws.nb_cnt + (size_t)p * 16 + (angular ? 8 : 0);
  int n = 0;
  for (int s = 0; s < 8; ++s) n += hdr[s];
  const int* lst = angular ? ws.nb_a + (size_t)p * ws.cap_a : ws.nb_r + (size_t)p * ws.cap_r;
  const int gi = ws.pos_src[p];
  for (int t = threadIdx.x; t < cap_out; t += blockDim.x)
    out[(size_t)gi * cap_out + t] = t < n ? ws.pos_src[lst[t]] : -1;
}

}  // namespace

void launch_finalize_e(const Ws& ws, int n_in, const float* e_row, int E, int e_row_net,
                       const double* ebias, cudaStream_t st) {
  if (n_in <= 0) return;
  k_finalize<<<(n_in + 255) / 256, 256, 0, st>>>(ws, e_row, E, e_row_net, ebias);
}

void launch_gather_rows(const Ws& ws, int n_in, const float* rows, const uint16_t* rows_h,
                        const uint16_t* rows_l, int ld, int D, const int16_t* col, float* out,
                        int by_tile, cudaStream_t st) {
  if (n_in <= 0) return;
  k_gather_rows<<<n_in, 128, 0, st>>>(ws, rows, rows_h, rows_l, ld, D, col, out, by_tile);
}

void launch_gather_nbrs(const Ws& ws, int n_in, int angular, int cap_out, int* out,
                        cudaStream_t st) {
  if (n_in <= 0) return;
  k_gather_nbrs<<<n_in, 128, 0, st>>>(ws, angular, cap_out, out);
}

}  // namespace nnp
