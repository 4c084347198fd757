// Internal declarations shared by the CUDA translation units of libnnp.
// Device-side layout of the work arena and the per-system descriptors.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nnp {

constexpr int kMaxSpecies = 8;
constexpr int kNR = 16;            // radial shells (Eq. 4)
constexpr int kNA = 4;             // angular distance shells (Eq. 5)
constexpr int kNZ = 8;             // angular sections (Eq. 5)
constexpr int kRowTile = 128;      // species segments of AEV rows are padded to this
constexpr int kMaxBatchParam = 64; // systems per kernel-parameter chunk
constexpr int kStageCap = 512;     // staged radial neighbours per centre (hard cap)

// status word bits (device)
enum : int {
  kStSpecies = 1,
  kStNonFinite = 2,
  kStCapacity = 4,
  kStCells = 8,
  kStTimeout = 16,
  kStBounds = 32,    // a checked index was out of range (bounds-checked builds only)
};

// ---- index checks of the bounds-checked build (-DNNP_DEBUG_BOUNDS, built as
// libnnp_debug.so).  A failed check sets kStBounds in the status word, records
// the first failing site in status[3] and makes the caller skip the access;
// the host turns it into NNP_ERR_BOUNDS.  In the normal build NNP_IN_BOUNDS is
// `true` and its arguments are not evaluated.
enum BoundsSite : int {
  kSiteNone = 0,
  kSiteBinCell,          // cell binning: global cell index < cell capacity
  kSiteScatterPos,       // scatter: packed position < batch atoms
  kSiteNbCandidate,      // neighbour search: list entry < ML atoms
  kSiteAevNeighbour,     // AEV kernels: staged neighbour < ML atoms
  kSiteAevRow,           // AEV forward: row slot < row capacity
  kSiteBwdNeighbour,     // AEV backward: force target < ML atoms
  kSiteBwdTriplet,       // AEV backward: triplet's neighbour slots < list length
  kSiteBwdHeavy,         // AEV backward: dense-centre list index < batch atoms
  kSiteFinalize,         // finalize: row slot < row capacity
  kSiteGemmRow,          // tensor-core epilogue: output row < row capacity
  kSiteCount
};

__host__ __device__ inline bool bounds_ok(int* status, int site, long long i, long long n) {
  if (i >= 0 && i < n) return true;
#ifdef __CUDA_ARCH__
  atomicOr(status, kStBounds);
  atomicCAS(status + 3, 0, site);
#else
  status[0] |= kStBounds;
  if (status[3] == 0) status[3] = site;
#endif
  return false;
}

#ifdef NNP_DEBUG_BOUNDS
#define NNP_IN_BOUNDS(status, site, i, n) \
  ::nnp::bounds_ok((status), (site), (long long)(i), (long long)(n))
constexpr bool kBoundsChecked = true;
#else
#define NNP_IN_BOUNDS(status, site, i, n) true
constexpr bool kBoundsChecked = false;
#endif

// AEV hyper-parameters in the form the kernels use
struct AevConst {
  int S;            // species
  int D;            // AEV length
  int Dp;           // padded row stride (multiple of 64)
  int n_pairs;      // S(S+1)/2
  float rc_r, rc_a, eta_r, eta_a;
  float shf_r[kNR];
  float shf_a[kNA];
  float cos_z[kNZ], sin_z[kNZ];
  float cos_scale;
  int zeta;         // integer exponent
  float ang_pre;    // 2^(1-zeta)
  float skin;       // Verlet skin of the neighbour lists (0: lists at the cutoffs)
  // Column layout of an AEV row: each block holds the paper's values, but the
  // blocks are stored in an order that puts those of common species first
  // (nnp_create fixes it from the atomic numbers); rcol[s]: first column of
  // radial block s, acol[q]: first column of angular block q (species pair q in
  // the paper's order).  Every block starts at a multiple of 16.
  int16_t rcol[kMaxSpecies];
  int16_t acol[kMaxSpecies * (kMaxSpecies + 1) / 2];
};

// per-system descriptor as passed in kernel parameters (host-filled part)
struct SysIn {
  const float* coords;
  const uint8_t* species;
  const uint8_t* mask;
  double* energy;
  float* forces;
  double* virial;
  float* atom_e;
  int n_in;
  int in_base;       // offset of this system's atoms in the batch input index space
  int periodic;
  float box_hi[3], box_lo[3];   // box edge as float hi + float residual
  float inv_box[3];             // 1 / box_hi (FP32), for the minimum-image shift
  // force vector-Jacobian product only (null otherwise)
  const float* dLdF;
  float* dLdR;
  double gE;
};

// per-system device state (device-filled part)
struct SysDev {
  SysIn in;
  int n_ml;          // atoms inside the mask
  int atom_base;     // first packed (cell-ordered) position of this system
  int cell_base;     // first global cell index
  int nc[3];         // cells per dimension
  float origin[3];   // cell grid origin (non-periodic: bounding-box minimum)
  float inv_cell[3]; // cells per Angstrom
  unsigned bb_min[3], bb_max[3];  // bounding box as order-preserving uint keys
};

struct BatchParams {
  int n_sys;         // systems in this chunk
  int sys_base;      // index of the first system of the chunk in the batch
  SysIn sys[kMaxBatchParam];
};

// device work arena (all pointers device)
struct Ws {
  int* status;       // [4]: flags, max radial count, max angular count, spare
  SysDev* sys;       // [max_sys]
  int n_sys;
  int n_in;          // batch input atoms (sum of n_in)
  int cell_cap;      // capacity of the global cell arrays
  int row_cap;       // capacity of AEV rows (n_in + S*kRowTile)
  int cap_r, cap_a;  // neighbour capacity per centre
  // counters
  int* species_count;   // [kMaxSpecies]
  int* species_fill;    // [kMaxSpecies]
  int* seg_start;       // [kMaxSpecies+1] 128-aligned row segments; [S] = total rows
  int* totals;          // [8]: total ML atoms, total cells, dense centres, -, next centre
                        // of the AEV forward and of the warp-per-centre backward
  int* cell_count;      // [cell_cap]
  int* cell_start;      // [cell_cap + 1]
  // per input atom
  int* in_cell;         // global cell or -1
  int* in_rank;
  int* in_slot;
  int* in_sys;
  // per packed (cell-ordered) atom
  float4* xyzq;         // x, y, z, species (int bits)
  int* pos_src;         // batch input index
  int* pos_slot;        // AEV row
  int* pos_sys;
  int* pos_cell;        // local cell index within the system grid
  int* slot_pos;        // [row_cap] packed position of the atom of an AEV row (rows < a
                        // segment's atom count; written at every list build)
  // neighbour lists
  uint16_t* nb_cnt;     // [n_in][16]: radial count per species [0..7], angular [8..15]
  int* nb_r;            // [n_in][cap_r] packed positions, species-sorted
  int* nb_a;            // [n_in][cap_a]
  // AEV / gradient
  float* aev;           // [row_cap][Dp]
  uint16_t* aev_h;      // [row_cap][Dp] BF16 copy (bit patterns) for the tensor-core path, or null
  uint16_t* aev_l;      // [row_cap][Dp] split path: bf16(G - bf16(G)), or null
  // tensor-core paths: 64-column slices of the AEV rows that hold a nonzero
  // block (bit k = columns 64k .. 64k+63; bit 0 always set), per row and OR-ed
  // over each 128-row tile; null: every row is written in full
  uint32_t* row_mask;   // [row_cap]
  uint32_t* tile_mask;  // [row_cap / 128 + 1]
  float* dEdG;          // [row_cap][Dp]
  float* atom_e;        // [row_cap] per-row energy (mean over the ensemble, incl. shift)
  float4* f_pos;        // [n_in] forces on packed atoms
  int* heavy;           // [n_in] packed positions of the centres the warp-per-centre
                        // AEV backward hands on (count in totals[2])
  // deterministic mode (null otherwise): the force kernels write every
  // contribution to its own slot instead of adding it atomically, and fixed-order
  // gathers and reductions sum them (results bitwise repeatable)
  float4* fr_det;       // [n_in][cap_r] radial edge term on the neighbour of list slot t
  float4* fa_det;       // [n_in][cap_a] angular terms on the neighbour of list slot t
  float4* fs_det;       // [n_in] the centre's own force
  double* e_det;        // [n_in] atomic energy (FP64), by packed position
  double* v_det;        // [n_in][9] the centre's virial contribution
  // persistent neighbour lists with a skin (null skin_state: rebuilt every call)
  int* skin_state;      // [4]: max displacement (float bits), forced rebuild, builds, lists valid
  float half_skin;      // rebuild when an atom moved farther than this since the build
  float4* ref;          // [n_in] input coordinates at the last build
  int* in_pos;          // [n_in] packed position of an input atom at the last build (-1: none)
  uint16_t* nbs_cnt;    // [n_in][16] lists at the cutoffs + skin, as nb_cnt / nb_r / nb_a
  int* nbs_r;           // [n_in][cap_r]
  int* nbs_a;           // [n_in][cap_a]
};

// whether this call rebuilds the cell lists and neighbour lists
__device__ __forceinline__ bool lists_rebuild(const Ws& ws) {
  if (!ws.skin_state) return true;
  const volatile int* k = ws.skin_state;
  return k[1] != 0 || k[3] == 0 || __int_as_float(k[0]) > ws.half_skin;
}

// ---- launchers (nl.cu)
void launch_init_chunk(const Ws& ws, const BatchParams& bp, cudaStream_t st);
void launch_prep_atoms(const Ws& ws, const BatchParams& bp, int n_in_chunk, int S,
                       cudaStream_t st);
void launch_setup(const Ws& ws, const AevConst& ac, cudaStream_t st);
void launch_bin(const Ws& ws, int n_in, cudaStream_t st);
void launch_scan(const Ws& ws, cudaStream_t st);
void launch_scatter(const Ws& ws, int n_in, cudaStream_t st);
void launch_neighbors(const Ws& ws, int n_in, const AevConst& ac, cudaStream_t st);
void launch_skin_check(const Ws& ws, const BatchParams& bp, int n_in_chunk, cudaStream_t st);
// init + prep + setup + bin + scan + scatter of a one-chunk batch in one CTA
void launch_front(const Ws& ws, const BatchParams& bp, const AevConst& ac, int n_in,
                  cudaStream_t st);
// deterministic mode (ws.fr_det set): after a list build, the atoms of every cell
// in input order and the AEV rows of every species in packed order (both are
// otherwise taken by atomic counters)
void launch_det_order(const Ws& ws, int S, cudaStream_t st);
// deterministic mode: f_pos[j] = own term + the terms of j in its neighbours'
// lists, summed in list order
void launch_det_force_gather(const Ws& ws, int n_in, cudaStream_t st);
// deterministic mode: system energies (and virials) summed over their packed
// positions in order
void launch_det_reduce(const Ws& ws, int want_virial, cudaStream_t st);
// ---- aev.cu
void launch_aev_fwd(const Ws& ws, int n_in, const AevConst& ac, cudaStream_t st);
// sparse rows (ws.row_mask set): zero the slices of each row that its tile reads
// (tile mask) but the row itself left unwritten
void launch_aev_fill(const Ws& ws, const AevConst& ac, cudaStream_t st);
// AEV of 128-row species tiles computed into shared memory and fed straight to
// the first layer's tensor-core GEMM (BF16, one-network models); false if the
// tile does not fit or the model is outside what the kernel handles
bool aev_l1_supported(const Ws& ws, const AevConst& ac, int E, int h1);
void launch_aev_l1(const Ws& ws, const AevConst& ac, const void* w1_bf16, const float* b1,
                   void* H1, int h1, float alpha, cudaStream_t st);
cudaError_t aev_l1_ensure_smem(const Ws& ws, const AevConst& ac, int h1);
void launch_aev_bwd(const Ws& ws, int n_in, const AevConst& ac, int want_virial,
                    cudaStream_t st);
cudaError_t aev_ensure_smem(const Ws& ws);
size_t aev_fwd_smem(const Ws& ws);
size_t aev_bwd_smem(const Ws& ws, int n_pairs = kMaxSpecies * (kMaxSpecies + 1) / 2);
// ---- finalize.cu
void launch_finalize_e(const Ws& ws, int n_in, const float* e_row, int E, int e_row_net,
                       const double* ebias, cudaStream_t st);
void launch_gather_rows(const Ws& ws, int n_in, const float* rows, const uint16_t* rows_h,
                        const uint16_t* rows_l, int ld, int D, const int16_t* col, float* out,
                        int by_tile, cudaStream_t st);
void launch_gather_nbrs(const Ws& ws, int n_in, int angular, int cap_out, int* out,
                        cudaStream_t st);

// Cells per dimension of one system's grid: edge >= rc (nc[c] <= len[c] / rc)
// and nc[0] nc[1] nc[2] <= cap.  Each count starts at floor(len / rc), clamped to
// [1, 2^20] (a non-finite or huge extent cannot overflow the product, which
// stays below 2^60); while the product exceeds cap the largest count is cut to
// cap / (product of the other two), at least 1, so the loop ends within three
// passes.  Returns the product.
__host__ __device__ inline long long cell_grid(const float len[3], float rc, long long cap,
                                               int nc[3]) {
  for (int c = 0; c < 3; ++c) {
    const float q = len[c] / rc;
    nc[c] = (q >= 1048576.f) ? 1048576 : (q >= 1.f ? (int)q : 1);   // NaN -> 1
  }
  long long prod = (long long)nc[0] * nc[1] * nc[2];
  while (prod > cap) {
    const int c = (nc[0] >= nc[1] && nc[0] >= nc[2]) ? 0 : (nc[1] >= nc[2] ? 1 : 2);
    const long long rest = prod / nc[c];
    const long long want = cap / rest;
    nc[c] = (int)(want < 1 ? 1 : want);
    prod = (long long)nc[0] * nc[1] * nc[2];
  }
  return prod;
}

// order-preserving float <-> uint key (for atomicMin/atomicMax on floats)
__host__ __device__ inline unsigned float_key(float f) {
  unsigned u;
#ifdef __CUDA_ARCH__
  u = __float_as_uint(f);
#else
  union { float f; unsigned u; } c; c.f = f; u = c.u;
#endif
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float key_float(unsigned k) {
  unsigned u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  union { float f; unsigned u; } c; c.u = u; return c.f;
#endif
}

}  // namespace nnp
