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
    if (ws.e_det) ws.e_det[p] = Ei;   // deterministic mode: summed in order later
  }
  if (ws.e_det) return;
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

// deterministic mode: f_pos[j] = j's own term + the terms of j that its
// neighbours i wrote into their list slots (found by scanning i's list for j:
// the lists are symmetric), each lane summing its neighbours in list order and
// the warp combining the lanes in a fixed tree
__global__ void k_det_force_gather(Ws ws) {
  const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
  const unsigned lane = threadIdx.x & 31;
  if (j >= ws.totals[0]) return;
  const uint16_t* hj = ws.nb_cnt + (size_t)j * 16;
  int nr = 0, na = 0;
  for (int s = 0; s < 8; ++s) { nr += hj[s]; na += hj[8 + s]; }
  float r[3] = {0.f, 0.f, 0.f}, a[3] = {0.f, 0.f, 0.f};
  for (int t = lane; t < nr; t += 32) {
    const int i = ws.nb_r[(size_t)j * ws.cap_r + t];
    if (!NNP_IN_BOUNDS(ws.status, kSiteBwdNeighbour, i, ws.totals[0])) continue;
    const uint16_t* hi = ws.nb_cnt + (size_t)i * 16;
    int ni = 0;
    for (int s = 0; s < 8; ++s) ni += hi[s];
    const int* li = ws.nb_r + (size_t)i * ws.cap_r;
    for (int u = 0; u < ni; ++u)
      if (li[u] == j) {
        const float4 f = ws.fr_det[(size_t)i * ws.cap_r + u];
        r[0] += f.x; r[1] += f.y; r[2] += f.z;
        break;
      }
  }
  for (int t = lane; t < na; t += 32) {
    const int i = ws.nb_a[(size_t)j * ws.cap_a + t];
    if (!NNP_IN_BOUNDS(ws.status, kSiteBwdNeighbour, i, ws.totals[0])) continue;
    const uint16_t* hi = ws.nb_cnt + (size_t)i * 16;
    int ni = 0;
    for (int s = 0; s < 8; ++s) ni += hi[8 + s];
    const int* li = ws.nb_a + (size_t)i * ws.cap_a;
    for (int u = 0; u < ni; ++u)
      if (li[u] == j) {
        const float4 f = ws.fa_det[(size_t)i * ws.cap_a + u];
        a[0] += f.x; a[1] += f.y; a[2] += f.z;
        break;
      }
  }
  for (int o = 16; o > 0; o >>= 1)
    for (int k = 0; k < 3; ++k) {
      r[k] += __shfl_xor_sync(0xffffffffu, r[k], o);
      a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
    }
  if (lane == 0) {
    const float4 f = ws.fs_det[j];
    ws.f_pos[j] = make_float4(f.x + (r[0] + a[0]), f.y + (r[1] + a[1]), f.z + (r[2] + a[2]), 0.f);
  }
}

// deterministic mode: warp per system, its energy (and virial) summed over its
// packed positions in a fixed order
__global__ void k_det_reduce(Ws ws, int want_virial) {
  const int b = blockIdx.x * 8 + (threadIdx.x >> 5);
  const unsigned lane = threadIdx.x & 31;
  if (b >= ws.n_sys) return;
  const SysDev& d = ws.sys[b];
  const int beg = d.atom_base, end = d.atom_base + d.n_ml;
  double e = 0.0;
  for (int p = beg + (int)lane; p < end; p += 32) e += ws.e_det[p];
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if (lane == 0 && d.in.energy) d.in.energy[0] = e;
  if (want_virial && d.in.virial)
    for (int k = 0; k < 9; ++k) {
      double v = 0.0;
      for (int p = beg + (int)lane; p < end; p += 32) v += ws.v_det[(size_t)p * 9 + k];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) d.in.virial[k] = v;
    }
}

}  // namespace

void launch_det_force_gather(const Ws& ws, int n_in, cudaStream_t st) {
  if (!ws.fr_det || n_in <= 0) return;
  k_det_force_gather<<<(n_in + 7) / 8, 256, 0, st>>>(ws);
}

void launch_det_reduce(const Ws& ws, int want_virial, cudaStream_t st) {
  if (!ws.e_det || ws.n_sys <= 0) return;
  k_det_reduce<<<(ws.n_sys + 7) / 8, 256, 0, st>>>(ws, want_virial);
}

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
