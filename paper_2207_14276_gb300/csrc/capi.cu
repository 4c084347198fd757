// Host runtime and C ABI of libnnp (declared in include/nnp.h).
//
// A handle = shared device model (AEV constants + network weights in the
// layouts the kernels read) + its own bounded work arena.  The arena is one
// device allocation carved into the buffers of a batch, sized in proportion to
// the number of atoms (the paper's upfront bounded buffer); it only grows, and
// only between calls.  Every compute call enqueues the kernel chain on the
// caller's stream without host synchronisation.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/nnp.h"
#include "mlp.cuh"
#include "nnp_internal.cuh"
#include "vjp.cuh"

using namespace nnp;

namespace nnp {
void launch_gemm_fp32(const GemmArgs& g, int row_cap, cudaStream_t st);
int launch_mlp_tc(const Ws& ws, const MlpDims& md, const MlpWeights& mw, const MlpBufs& mb,
                  float alpha, cudaStream_t st, int* n_launch, StageHook* hook, void* state,
                  bool energy_only, bool skip_l1);
int mlp_tc_prepare(const MlpDims& md, const MlpWeights& mw, const MlpBufs& mb, int row_cap,
                   const float* aev, float* dEdG, bool split, void** state);
void mlp_tc_release(void* state);
void mlp_tc_use_chain(void* state, bool on);
void launch_aev_to_bf16(const Ws& ws, int n_in, const AevConst& ac, void* out, cudaStream_t st);
void launch_wait_probe(int* status, unsigned limit, cudaStream_t st);
}  // namespace nnp

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CU_TRY(x)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (x);                                                           \
    if (e_ != cudaSuccess)                                                          \
      return fail(NNP_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_));   \
  } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// how the per-species networks run
enum NetPath : int {
  kNetSimt = 0,    // FP32 FMA: the fused kernel (one network) or six SIMT GEMMs
  kNetBf16 = 1,    // tcgen05 GEMMs on BF16 operands
  kNetSplit = 2,   // tcgen05 GEMMs on split BF16 operands (hi + lo), FP32-accurate
};

struct Model {
  std::atomic<int> refs{1};
  int device = 0;
  int precision = NNP_FP32;
  int net = kNetSimt;
  AevConst ac{};
  MlpDims md{};
  float alpha = 0.1f;
  MlpWeights mw{};
  double* ebias = nullptr;  // device [S]
  std::vector<int16_t> col_of_feat;   // AEV column of each feature of the paper's order [D]
  int16_t* col_of_feat_dev = nullptr; // the same on the device
  int16_t* feat_of_col_dev = nullptr; // its inverse [D]
  std::vector<void*> allocs;
  ~Model() {
    for (void* p : allocs) cudaFree(p);
  }
};

}  // namespace

struct nnp_handle {
  Model* model = nullptr;
  size_t budget = 0;
  // arena
  void* arena = nullptr;
  size_t arena_bytes = 0;
  int cap_in = 0, cap_sys = 0, cap_r = 128, cap_a = 48;
  bool dirty = true;  // capacities changed: re-carve before the next call
  Ws ws{};
  MlpBufs mb{};
  int* status_host = nullptr;  // pinned: [4] status words, then out_host
  double* out_host = nullptr;  // pinned [10]: energy and virial of a host-buffer call
  int last_launches = 0;
  int last_n_in = 0;
  bool last_aev_fp32 = true;  // the last call wrote the FP32 AEV rows (else the BF16 planes)
  void* tc_state = nullptr;
  // host-call staging
  void* stage = nullptr;
  size_t stage_bytes = 0;
  // force vector-Jacobian product buffers (grown on demand)
  void* vjp_arena = nullptr;
  size_t vjp_bytes = 0;
  int vjp_rows = 0;
  VjpBufs vb{};
  // replay of a repeated call as a CUDA graph
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::string gsig;       // signature of the captured call
  std::string last_sig;   // signature of the previous eager call
  int last_launches_graph = 0;
  // tensor-core paths: the layers after the first as one fused kernel (off by
  // default: on the 100k-atom ensemble it ties with the four layer GEMMs on the
  // split path and is slower on BF16)
  bool fused_chain = false;
  // BF16 one-network models: the AEV computed into shared memory and fed to the
  // first layer in one kernel (off by default)
  bool fused_aev_l1 = false;
  bool last_aev_stored = true;   // the last call wrote AEV rows to the arena
  // tensor-core paths: AEV rows written only in their live 64-column slices, the
  // first and last layer GEMMs restricted to them (exact: the rest is zero)
  bool sparse_rows = true;
  bool last_sparse = false;      // the last call ran with sparse rows
  // deterministic mode: atoms and AEV rows in sorted order, force and energy
  // contributions in their own slots summed in a fixed order (bitwise repeatable)
  bool det = false;
  // persistent neighbour lists with a Verlet skin (0: rebuilt on every call)
  float skin = 0.f;
  bool lists_valid = false;   // the lists in the arena belong to list_sig's batch layout
  std::string list_sig;
  long long skin_calls = 0;
  // optional per-stage CUDA-event timing
  bool profile = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  double prof_ms[32] = {0};
  long long prof_calls[32] = {0};
};

namespace {

// ---------------------------------------------------------------- model setup
// Column layout of the AEV rows.  The paper lists the radial blocks species by
// species, then the angular blocks by species pair (s <= u, row-major).  The
// library keeps each block's values but stores the blocks ordered by how common
// their species are in solvated biomolecular systems (H, O, C, N, S, F, Cl, then
// by atomic number): a species' radial block, then its pairs with the species
// before it and with itself.  A water atom's row then holds all its nonzero
// values (radial H, O; angular HH, HO, OO) in its first 128 columns, so the
// sparse-row GEMMs skip most of the rest.  The first layer's weights are placed
// to match, and the diagnostic reads return the paper's order.
void aev_layout(AevConst& ac, const int* z, std::vector<int16_t>& col_of_feat) {
  const int S = ac.S;
  static const int kCommon[] = {1, 8, 6, 7, 16, 9, 17};
  auto rank = [&](int s) {
    for (int i = 0; i < 7; ++i)
      if (kCommon[i] == z[s]) return i;
    return 7 + std::max(z[s], 0);
  };
  struct Blk { int k0, k1, k2, angular, idx; };
  std::vector<Blk> blocks;
  for (int s = 0; s < S; ++s) blocks.push_back({rank(s), 0, 0, 0, s});
  for (int s = 0, q = 0; s < S; ++s)
    for (int u = s; u < S; ++u, ++q)
      blocks.push_back({std::max(rank(s), rank(u)), 1, std::min(rank(s), rank(u)), 1, q});
  std::stable_sort(blocks.begin(), blocks.end(), [](const Blk& x, const Blk& y) {
    return x.k0 != y.k0 ? x.k0 < y.k0 : x.k1 != y.k1 ? x.k1 < y.k1 : x.k2 < y.k2;
  });
  col_of_feat.assign(ac.D, 0);
  int c = 0;
  for (const Blk& b : blocks) {
    const int width = b.angular ? kNA * kNZ : kNR;
    const int f0 = b.angular ? S * kNR + b.idx * kNA * kNZ : b.idx * kNR;
    if (b.angular) ac.acol[b.idx] = (int16_t)c;
    else ac.rcol[b.idx] = (int16_t)c;
    for (int i = 0; i < width; ++i) col_of_feat[f0 + i] = (int16_t)(c + i);
    c += width;
  }
}

int build_model(Model* m, const nnp_species_t* sp, const nnp_aev_params_t* a,
                const nnp_weights_t* w, int precision) {
  if (!sp || !a || !w) return fail(NNP_ERR_ARG, "null argument");
  const int S = sp->n_species;
  if (S < 1 || S > kMaxSpecies) return fail(NNP_ERR_ARG, "n_species must be in [1, 8]");
  if (a->n_shf_r != kNR || a->n_shf_a != kNA || a->n_shf_z != kNZ)
    return fail(NNP_ERR_UNSUPPORTED, "kernels implement 16 radial, 4 angular-distance and 8 angle shells");
  const double zr = std::round((double)a->zeta);
  if (std::fabs(a->zeta - zr) > 0 || zr < 1 || zr > 64)
    return fail(NNP_ERR_UNSUPPORTED, "zeta must be an integer in [1, 64]");
  if (!(a->rc_r > 0) || !(a->rc_a > 0) || !(a->eta_r > 0) || !(a->eta_a > 0))
    return fail(NNP_ERR_ARG, "cutoffs and widths must be positive");
  if (a->rc_a > a->rc_r) return fail(NNP_ERR_UNSUPPORTED, "angular cutoff must not exceed the radial one");
  if (!(a->cos_scale > 0) || a->cos_scale > 1) return fail(NNP_ERR_ARG, "cos_scale must be in (0, 1]");
  if (w->n_layers != 4 || !w->widths || !w->params || w->n_ensemble < 1)
    return fail(NNP_ERR_UNSUPPORTED, "networks must have 4 layers");
  if (precision != NNP_FP32 && precision != NNP_BF16_MLP && precision != NNP_FP32_SPLIT &&
      precision != NNP_FP32_SIMT)
    return fail(NNP_ERR_ARG, "bad precision");
  AevConst& ac = m->ac;
  ac.S = S;
  ac.D = S * kNR + S * (S + 1) / 2 * kNA * kNZ;
  ac.Dp = (int)align_up(ac.D, 64);
  ac.n_pairs = S * (S + 1) / 2;
  ac.rc_r = a->rc_r; ac.rc_a = a->rc_a; ac.eta_r = a->eta_r; ac.eta_a = a->eta_a;
  for (int r = 0; r < kNR; ++r) ac.shf_r[r] = a->shf_r[r];
  for (int r = 0; r < kNA; ++r) ac.shf_a[r] = a->shf_a[r];
  for (int z = 0; z < kNZ; ++z) {
    ac.cos_z[z] = (float)std::cos((double)a->shf_z[z]);
    ac.sin_z[z] = (float)std::sin((double)a->shf_z[z]);
  }
  ac.cos_scale = a->cos_scale;
  ac.zeta = (int)zr;
  ac.ang_pre = (float)std::pow(2.0, 1.0 - zr);
  aev_layout(ac, sp->atomic_numbers, m->col_of_feat);
  const int* wd = w->widths;
  if (wd[0] != ac.D) return fail(NNP_ERR_ARG, "widths[0] must equal the AEV length");
  if (wd[4] != 1) return fail(NNP_ERR_ARG, "output width must be 1");
  for (int l = 1; l < 4; ++l)
    if (wd[l] < 16 || wd[l] % 16 != 0 || wd[l] > 512)
      return fail(NNP_ERR_UNSUPPORTED, "hidden widths must be multiples of 16 in [16, 512]");
  MlpDims& md = m->md;
  md.S = S; md.E = w->n_ensemble; md.Dp = ac.Dp; md.h1 = wd[1]; md.h2 = wd[2]; md.h3 = wd[3];
  m->alpha = w->celu_alpha;
  if (!(m->alpha > 0)) return fail(NNP_ERR_ARG, "celu_alpha must be positive");
  m->precision = precision;
  // FP32 accuracy: the split tensor-core path (measured faster than the FP32 FMA
  // kernels for ensembles and for one-network models alike)
  m->net = precision == NNP_BF16_MLP    ? kNetBf16
           : precision == NNP_FP32_SIMT ? kNetSimt
                                        : kNetSplit;
  CU_TRY(cudaGetDevice(&m->device));

  // unpack the flat parameter vector into the kernel layouts
  const int E = md.E, D = ac.D, Dp = ac.Dp, h1 = md.h1, h2 = md.h2, h3 = md.h3;
  std::vector<float> W1cat((size_t)S * E * h1 * Dp, 0.f), b1cat((size_t)S * E * h1);
  std::vector<float> W2((size_t)E * S * h2 * h1), b2((size_t)E * S * h2);
  std::vector<float> W3((size_t)E * S * h3 * h2), b3((size_t)E * S * h3);
  std::vector<float> w4((size_t)E * S * h3), W3T((size_t)E * S * h2 * h3);
  std::vector<float> W2T((size_t)E * S * h1 * h2), W1Tcat((size_t)S * Dp * E * h1, 0.f);
  std::vector<double> ebias(S, 0.0);
  const float* p = w->params;
  for (int e = 0; e < E; ++e)
    for (int s = 0; s < S; ++s) {
      const float* L1 = p; p += (size_t)h1 * D;
      const float* B1 = p; p += h1;
      const float* L2 = p; p += (size_t)h2 * h1;
      const float* B2 = p; p += h2;
      const float* L3 = p; p += (size_t)h3 * h2;
      const float* B3 = p; p += h3;
      const float* L4 = p; p += h3;
      const float* B4 = p; p += 1;
      for (int o = 0; o < h1; ++o) {
        for (int k = 0; k < D; ++k) {
          const int c = m->col_of_feat[k];   // feature k of the paper's order
          W1cat[((size_t)s * E * h1 + e * h1 + o) * Dp + c] = L1[(size_t)o * D + k];
          W1Tcat[((size_t)s * Dp + c) * E * h1 + e * h1 + o] = L1[(size_t)o * D + k] / (float)E;
        }
        b1cat[(size_t)s * E * h1 + e * h1 + o] = B1[o];
      }
      const size_t es = (size_t)e * S + s;
      for (int o = 0; o < h2; ++o) {
        for (int k = 0; k < h1; ++k) {
          W2[(es * h2 + o) * h1 + k] = L2[(size_t)o * h1 + k];
          W2T[(es * h1 + k) * h2 + o] = L2[(size_t)o * h1 + k];
        }
        b2[es * h2 + o] = B2[o];
      }
      for (int o = 0; o < h3; ++o) {
        for (int k = 0; k < h2; ++k) {
          W3[(es * h3 + o) * h2 + k] = L3[(size_t)o * h2 + k];
          W3T[(es * h2 + k) * h3 + o] = L3[(size_t)o * h2 + k];
        }
        b3[es * h3 + o] = B3[o];
        w4[es * h3 + o] = L4[o];
      }
      ebias[s] += (double)B4[0] / E;
    }
  for (int s = 0; s < S; ++s)
    if (w->species_shift) ebias[s] += w->species_shift[s];

  auto upload = [&](const void* src, size_t bytes, void** dst) -> int {
    CU_TRY(cudaMalloc(dst, bytes));
    m->allocs.push_back(*dst);
    CU_TRY(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    return NNP_OK;
  };
  auto upf = [&](const std::vector<float>& v, float** dst) {
    return upload(v.data(), v.size() * sizeof(float), reinterpret_cast<void**>(dst));
  };
  int rc;
  if ((rc = upf(W1cat, &m->mw.W1cat))) return rc;
  if ((rc = upf(b1cat, &m->mw.b1cat))) return rc;
  if ((rc = upf(W2, &m->mw.W2))) return rc;
  if ((rc = upf(b2, &m->mw.b2))) return rc;
  if ((rc = upf(W3, &m->mw.W3))) return rc;
  if ((rc = upf(b3, &m->mw.b3))) return rc;
  if ((rc = upf(w4, &m->mw.w4))) return rc;
  if ((rc = upf(W3T, &m->mw.W3T))) return rc;
  if ((rc = upf(W2T, &m->mw.W2T))) return rc;
  if ((rc = upf(W1Tcat, &m->mw.W1Tcat))) return rc;
  if ((rc = upload(ebias.data(), S * sizeof(double), reinterpret_cast<void**>(&m->ebias)))) return rc;
  std::vector<int16_t> feat_of_col(D);
  for (int k = 0; k < D; ++k) feat_of_col[m->col_of_feat[k]] = (int16_t)k;
  if ((rc = upload(m->col_of_feat.data(), D * sizeof(int16_t),
                   reinterpret_cast<void**>(&m->col_of_feat_dev))))
    return rc;
  if ((rc = upload(feat_of_col.data(), D * sizeof(int16_t),
                   reinterpret_cast<void**>(&m->feat_of_col_dev))))
    return rc;
  if (m->net != kNetSimt) {
    // BF16 copies of the GEMM operands (round to nearest even); the split path
    // also keeps the rounded remainders w - bf16(w)
    auto bf16_bits = [](float x) {
      uint32_t u;
      std::memcpy(&u, &x, 4);
      return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
    };
    auto bf16_value = [](uint16_t b) {
      const uint32_t u = (uint32_t)b << 16;
      float x;
      std::memcpy(&x, &u, 4);
      return x;
    };
    auto upb = [&](const std::vector<float>& v, void** hi, void** lo) {
      std::vector<uint16_t> h(v.size()), l(lo ? v.size() : 0);
      for (size_t i = 0; i < v.size(); ++i) {
        h[i] = bf16_bits(v[i]);
        if (lo) l[i] = bf16_bits(v[i] - bf16_value(h[i]));
      }
      int r = upload(h.data(), h.size() * sizeof(uint16_t), hi);
      if (r == NNP_OK && lo) r = upload(l.data(), l.size() * sizeof(uint16_t), lo);
      return r;
    };
    const bool sp = m->net == kNetSplit;
    MlpWeights& mw = m->mw;
    if ((rc = upb(W1cat, &mw.W1cat_h, sp ? &mw.W1cat_l : nullptr))) return rc;
    if ((rc = upb(W2, &mw.W2_h, sp ? &mw.W2_l : nullptr))) return rc;
    if ((rc = upb(W3, &mw.W3_h, sp ? &mw.W3_l : nullptr))) return rc;
    if ((rc = upb(W3T, &mw.W3T_h, sp ? &mw.W3T_l : nullptr))) return rc;
    if ((rc = upb(W2T, &mw.W2T_h, sp ? &mw.W2T_l : nullptr))) return rc;
    if ((rc = upb(W1Tcat, &mw.W1Tcat_h, sp ? &mw.W1Tcat_l : nullptr))) return rc;
  }
  return NNP_OK;
}

// ---------------------------------------------------------------- arena
struct Carve {
  char* base;
  size_t off = 0;
  template <class T> T* take(size_t n) {
    off = align_up(off, 256);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};

size_t carve(nnp_handle* h, char* base) {
  const Model& m = *h->model;
  const int S = m.ac.S, Dp = m.ac.Dp, E = m.md.E;
  const size_t n = std::max(h->cap_in, 1);
  const size_t nsys = std::max(h->cap_sys, 1);
  const size_t cells = 2 * n + 27 * nsys;
  const size_t rows = n + (size_t)S * kRowTile;
  Carve c{base};
  Ws& ws = h->ws;
  ws.status = c.take<int>(4);
  ws.sys = c.take<SysDev>(nsys);
  ws.cell_cap = (int)cells;
  ws.row_cap = (int)rows;
  ws.cap_r = h->cap_r;
  ws.cap_a = h->cap_a;
  ws.species_count = c.take<int>(kMaxSpecies);
  ws.species_fill = c.take<int>(kMaxSpecies);
  ws.seg_start = c.take<int>(kMaxSpecies + 1);
  ws.totals = c.take<int>(8);
  ws.cell_count = c.take<int>(cells);
  ws.cell_start = c.take<int>(cells + 1);
  ws.in_cell = c.take<int>(n);
  ws.in_rank = c.take<int>(n);
  ws.in_slot = c.take<int>(n);
  ws.in_sys = c.take<int>(n);
  ws.xyzq = c.take<float4>(n);
  ws.pos_src = c.take<int>(n);
  ws.pos_slot = c.take<int>(n);
  ws.pos_sys = c.take<int>(n);
  ws.pos_cell = c.take<int>(n);
  ws.slot_pos = c.take<int>(rows);
  ws.nb_cnt = c.take<uint16_t>(n * 16);
  ws.nb_r = c.take<int>(n * h->cap_r);
  ws.nb_a = c.take<int>(n * h->cap_a);
  ws.aev = c.take<float>(rows * Dp);
  ws.dEdG = c.take<float>(rows * Dp);
  ws.atom_e = c.take<float>(rows);
  ws.f_pos = c.take<float4>(n);
  ws.heavy = c.take<int>(n);
  if (h->det) {
    ws.fr_det = c.take<float4>(n * h->cap_r);
    ws.fa_det = c.take<float4>(n * h->cap_a);
    ws.fs_det = c.take<float4>(n);
    ws.e_det = c.take<double>(n);
    ws.v_det = c.take<double>(n * 9);
  } else {
    ws.fr_det = ws.fa_det = ws.fs_det = nullptr;
    ws.e_det = ws.v_det = nullptr;
  }
  if (h->skin > 0.f) {
    ws.skin_state = c.take<int>(4);
    ws.ref = c.take<float4>(n);
    ws.in_pos = c.take<int>(n);
    ws.nbs_cnt = c.take<uint16_t>(n * 16);
    ws.nbs_r = c.take<int>(n * h->cap_r);
    ws.nbs_a = c.take<int>(n * h->cap_a);
  } else {
    ws.skin_state = nullptr;
    ws.ref = nullptr;
    ws.in_pos = nullptr;
    ws.nbs_cnt = nullptr;
    ws.nbs_r = nullptr;
    ws.nbs_a = nullptr;
  }
  ws.half_skin = 0.5f * h->skin;
  const bool tc = (m.net != kNetSimt), split = (m.net == kNetSplit);
  const size_t esz = tc ? 2 : 4;
  MlpBufs& mb = h->mb;
  mb = MlpBufs{};
  // the fused FP32 kernel keeps its activations on chip; the tensor-core paths
  // rebuild CELU' from the activations and store no derivative buffers; the
  // split path stores every activation as two BF16 planes (high, low)
  if (tc || !mlp_fused_supported(m.md)) {
    mb.H1 = c.take<char>(rows * E * m.md.h1 * esz);
    mb.H2 = c.take<char>(rows * E * m.md.h2 * esz);
    mb.d3 = c.take<char>(rows * E * m.md.h3 * esz);
    if (!tc) {
      mb.D1 = c.take<char>(rows * E * m.md.h1 * esz);
      mb.D2 = c.take<char>(rows * E * m.md.h2 * esz);
    }
    if (split) {
      mb.H1l = c.take<char>(rows * E * m.md.h1 * 2);
      mb.H2l = c.take<char>(rows * E * m.md.h2 * 2);
      mb.d3l = c.take<char>(rows * E * m.md.h3 * 2);
    }
  }
  mb.e_row = c.take<float>((size_t)E * rows);
  mb.aev_h = tc ? c.take<char>(rows * Dp * 2) : nullptr;
  mb.aev_l = split ? c.take<char>(rows * Dp * 2) : nullptr;
  ws.aev_h = static_cast<uint16_t*>(mb.aev_h);
  ws.aev_l = static_cast<uint16_t*>(mb.aev_l);
  // tensor-core paths: rows written only in their live slices (the first layer
  // reads a tile's live slices, the last backward layer computes only those)
  ws.row_mask = tc ? c.take<uint32_t>(rows) : nullptr;
  ws.tile_mask = tc ? c.take<uint32_t>(rows / kRowTile + 1) : nullptr;
  return align_up(c.off, 256);
}

int ensure_arena(nnp_handle* h, int n_in, int n_sys) {
  if (!h->dirty && n_in <= h->cap_in && n_sys <= h->cap_sys) return NNP_OK;
  int want_in = std::max(n_in, h->cap_in), want_sys = std::max(n_sys, h->cap_sys);
  if (n_in > h->cap_in) want_in = std::max(n_in, (int)std::min<long long>(1LL << 30, (long long)h->cap_in * 5 / 4));
  if (n_sys > h->cap_sys) want_sys = std::max(n_sys, h->cap_sys * 5 / 4);
  const int old_in = h->cap_in, old_sys = h->cap_sys;
  h->cap_in = want_in;
  h->cap_sys = want_sys;
  const size_t bytes = carve(h, nullptr);
  if (h->budget && bytes > h->budget) {
    h->cap_in = old_in;
    h->cap_sys = old_sys;
    carve(h, static_cast<char*>(h->arena));
    return fail(NNP_ERR_OOM, "work arena of " + std::to_string(bytes) + " bytes exceeds the HBM budget");
  }
  if (h->arena) {
    CU_TRY(cudaDeviceSynchronize());
    if (h->tc_state) { mlp_tc_release(h->tc_state); h->tc_state = nullptr; }
    cudaFree(h->arena);
    h->arena = nullptr;
  }
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    h->cap_in = 0;
    h->cap_sys = 0;
    h->dirty = true;
    return fail(NNP_ERR_OOM, "cudaMalloc of the work arena (" + std::to_string(bytes) + " bytes) failed");
  }
  CU_TRY(cudaMemset(p, 0, bytes));
  h->arena = p;
  h->arena_bytes = bytes;
  h->lists_valid = false;
  carve(h, static_cast<char*>(p));
  // raise-only: other handles of the process may need larger limits
  CU_TRY(aev_ensure_smem(h->ws));
  CU_TRY(mlp_fused_ensure_smem(h->model->md));
  if (h->model->net != kNetSimt) {
    int rc = mlp_tc_prepare(h->model->md, h->model->mw, h->mb, h->ws.row_cap, h->ws.aev,
                            h->ws.dEdG, h->model->net == kNetSplit, &h->tc_state);
    if (rc) return fail(rc, "tensor-core GEMM set-up (tensor maps, launch limits) failed");
    mlp_tc_use_chain(h->tc_state, h->fused_chain);
    if (h->model->md.E == 1) CU_TRY(aev_l1_ensure_smem(h->ws, h->model->ac, h->model->md.h1));
  }
  h->dirty = false;
  return NNP_OK;
}

// stage names (index = stage id) reported by nnp_profile_read
const char* kStageNames[] = {"prep", "neighbors", "aev_fwd", "mlp_l1", "mlp_l2", "mlp_l3",
                             "mlp_b3", "mlp_b2", "mlp_b1", "aev_bwd", "finalize", "mlp_cvt",
                             "mlp", "mlp_chain", "aev_l1"};
constexpr int kNumStages = 15;

cudaEvent_t prof_event(nnp_handle* h) {
  if (!h->prof_pool.empty()) {
    cudaEvent_t e = h->prof_pool.back();
    h->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// brackets the kernels of one stage with events on the launching stream
struct StageTimer {
  nnp_handle* h;
  cudaStream_t st;
  int id;
  cudaEvent_t a = nullptr;
  StageTimer(nnp_handle* h_, cudaStream_t st_, int id_) : h(h_), st(st_), id(id_) {
    if (h->profile) { a = prof_event(h); cudaEventRecord(a, st); }
  }
  ~StageTimer() {
    if (h->profile) {
      cudaEvent_t b = prof_event(h);
      cudaEventRecord(b, st);
      h->prof_pending.push_back({id, {a, b}});
    }
  }
};

}  // namespace

namespace nnp {
void StageHook::begin(int id) {
  nnp_handle* hh = static_cast<nnp_handle*>(h);
  if (!hh->profile) return;
  cudaEvent_t ev = prof_event(hh);
  cudaEventRecord(ev, static_cast<cudaStream_t>(st));
  cur = ev;
  cur_id = id;
}
void StageHook::end() {
  nnp_handle* hh = static_cast<nnp_handle*>(h);
  if (!hh->profile || !cur) return;
  cudaEvent_t b = prof_event(hh);
  cudaEventRecord(b, static_cast<cudaStream_t>(st));
  hh->prof_pending.push_back({cur_id, {static_cast<cudaEvent_t>(cur), b}});
  cur = nullptr;
}
}  // namespace nnp

namespace {

void split_box(double L, float* hi, float* lo, float* inv) {
  *hi = (float)L;
  *lo = (float)(L - (double)*hi);
  *inv = 1.f / *hi;
}

// batches up to this many atoms (in one descriptor chunk) run the front end of
// the chain in one CTA
constexpr int kFrontMaxAtoms = 2048;

// the kernel chain of one batch on stream st (no host synchronisation)
int enqueue_batch(nnp_handle* h, int n_sys, const nnp_system_t* sy, const std::vector<BatchParams>& chunks,
                  int n_in, bool any_virial, cudaStream_t st, int* n_launch) {
  const Model& m = *h->model;
  Ws& ws = h->ws;
  int launches = 0, rc = NNP_OK;
  // systems without atoms: the outputs are the empty sums
  for (int b = 0; b < n_sys; ++b)
    if (sy[b].n_atoms == 0) {
      CU_TRY(cudaMemsetAsync(sy[b].energy, 0, sizeof(double), st));
      if (sy[b].virial) CU_TRY(cudaMemsetAsync(sy[b].virial, 0, 9 * sizeof(double), st));
      launches += 1 + (sy[b].virial ? 1 : 0);
    }
  // persistent lists: the displacement check decides on the device whether this
  // call rebuilds them (a new batch layout or a capacity change always does)
  AevConst ac = m.ac;
  ac.skin = ws.skin_state ? h->skin : 0.f;
  // a launch that fails is reported with the name of its stage
  auto chk = [&](const char* name) -> int {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NNP_OK : fail(NNP_ERR_CUDA, std::string(name) + ": " + cudaGetErrorString(e));
  };
  if (ws.skin_state) {
    const bool forced = !h->lists_valid;
    CU_TRY(cudaMemsetAsync(ws.skin_state, 0, sizeof(int), st));
    CU_TRY(cudaMemsetAsync(ws.skin_state + 1, forced ? 1 : 0, sizeof(int), st));
    launches += 2;
    if (!forced)
      for (const auto& bp : chunks) {
        int n_chunk = 0;
        for (int k = 0; k < bp.n_sys; ++k) n_chunk += bp.sys[k].n_in;
        if (n_chunk > 0) { launch_skin_check(ws, bp, n_chunk, st); ++launches; }
      }
    if ((rc = chk("displacement check"))) return rc;
  }
  // small one-chunk batches: the whole front end in one single-CTA launch
  const bool one_cta_front = chunks.size() == 1 && n_in > 0 && n_in <= kFrontMaxAtoms &&
                             !ws.skin_state;
  if (one_cta_front) {
    StageTimer t(h, st, 0);
    launch_front(ws, chunks[0], ac, n_in, st);
    ++launches;
  } else {
    for (const auto& bp : chunks) { launch_init_chunk(ws, bp, st); ++launches; }
    for (const auto& bp : chunks) {
      int n_chunk = 0;
      for (int k = 0; k < bp.n_sys; ++k) n_chunk += bp.sys[k].n_in;
      if (n_chunk > 0) { launch_prep_atoms(ws, bp, n_chunk, m.ac.S, st); ++launches; }
    }
  }
  if ((rc = chk("init/prep"))) return rc;
  if (n_in > 0) {
    if (!one_cta_front) {
      StageTimer t(h, st, 0);
      launch_setup(ws, ac, st);
      launch_bin(ws, n_in, st);
      launch_scan(ws, st);
      launch_scatter(ws, n_in, st);
      launches += 4;
    }
    if ((rc = chk("cell lists"))) return rc;
    if (ws.fr_det) {   // deterministic mode: sorted atoms and rows
      StageTimer t(h, st, 0);
      launch_det_order(ws, m.ac.S, st);
      launches += 2;
    }
    { StageTimer t(h, st, 1); launch_neighbors(ws, n_in, ac, st); }
    if ((rc = chk("neighbors"))) return rc;
    if (ws.skin_state) ++launches;   // the list refresh
    const bool fuse_l1 = h->fused_aev_l1 && m.net == kNetBf16 &&
                         aev_l1_supported(ws, ac, m.md.E, m.md.h1);
    h->last_aev_stored = !fuse_l1;
    // sparse rows where the networks run on the tensor cores (ws.row_mask set)
    Ws wa = ws;
    if (!h->sparse_rows || fuse_l1) { wa.row_mask = nullptr; wa.tile_mask = nullptr; }
    h->last_sparse = wa.row_mask != nullptr;
    if (fuse_l1) {
      StageTimer t(h, st, 14);
      launch_aev_l1(ws, ac, m.mw.W1cat_h, m.mw.b1cat, h->mb.H1, m.md.h1, m.alpha, st);
    } else {
      StageTimer t(h, st, 2);
      launch_aev_fwd(wa, n_in, ac, st);
      if (wa.row_mask) { launch_aev_fill(wa, ac, st); ++launches; }
    }
    if ((rc = chk("aev_fwd"))) return rc;
    launches += 2;
    // energy only when no system asks for forces or a virial
    bool energy_only = true;
    for (int b = 0; b < n_sys; ++b) energy_only &= (sy[b].forces == nullptr && sy[b].virial == nullptr);
    StageHook hook{h, st};
    if (m.net != kNetSimt) {
      rc = launch_mlp_tc(wa, m.md, m.mw, h->mb, m.alpha, st, &launches, &hook, h->tc_state, energy_only,
                         fuse_l1);
      if (rc) return rc;
    } else {
      launch_mlp_fp32(ws, m.md, m.mw, h->mb, m.alpha, st, &launches, &hook, energy_only);
    }
    if ((rc = chk("mlp"))) return rc;
    if (!energy_only) {
      StageTimer t(h, st, 9);
      launch_aev_bwd(ws, n_in, ac, any_virial ? 1 : 0, st);
      if (ws.fr_det) { launch_det_force_gather(ws, n_in, st); ++launches; }
    }
    if ((rc = chk("aev_bwd"))) return rc;
    {
      StageTimer t(h, st, 10);
      launch_finalize_e(ws, n_in, h->mb.e_row, m.md.E, ws.row_cap, m.ebias, st);
      if (ws.e_det) { launch_det_reduce(ws, any_virial ? 1 : 0, st); ++launches; }
    }
    launches += 2;
  }
  CU_TRY(cudaGetLastError());
  *n_launch = launches;
  return rc;
}

// enqueue the whole chain for a batch whose descriptors are already validated
int run_batch(nnp_handle* h, int n_sys, const nnp_system_t* sy, cudaStream_t st) {
  const Model& m = *h->model;
  long long n_in_ll = 0;
  for (int b = 0; b < n_sys; ++b) n_in_ll += sy[b].n_atoms;
  if (n_in_ll > (1LL << 30)) return fail(NNP_ERR_ARG, "too many atoms in one call");
  const int n_in = (int)n_in_ll;
  int rc = ensure_arena(h, n_in, n_sys);
  if (rc) return rc;
  Ws& ws = h->ws;
  ws.n_sys = n_sys;
  ws.n_in = n_in;
  h->last_aev_fp32 = (m.net == kNetSimt);
  // per-chunk descriptors as kernel parameters
  std::vector<BatchParams> chunks;
  int in_base = 0;
  for (int b0 = 0; b0 < n_sys; b0 += kMaxBatchParam) {
    BatchParams bp{};
    bp.sys_base = b0;
    bp.n_sys = std::min(kMaxBatchParam, n_sys - b0);
    for (int k = 0; k < bp.n_sys; ++k) {
      const nnp_system_t& s = sy[b0 + k];
      SysIn& si = bp.sys[k];
      si.coords = s.coords;
      si.species = s.species;
      si.mask = s.mask;
      si.energy = s.energy;
      si.forces = s.forces;
      si.virial = s.virial;
      si.atom_e = s.atom_energies;
      si.n_in = (int)s.n_atoms;
      si.in_base = in_base;
      si.periodic = s.periodic ? 1 : 0;
      for (int c = 0; c < 3; ++c) split_box(s.periodic ? s.box[c] : 1.0, &si.box_hi[c], &si.box_lo[c], &si.inv_box[c]);
      in_base += (int)s.n_atoms;
    }
    chunks.push_back(bp);
  }
  bool any_virial = false;
  for (int b = 0; b < n_sys; ++b) any_virial |= (sy[b].virial != nullptr);
  if (ws.skin_state) {
    // the lists persist while the batch layout (sizes, species and mask arrays,
    // boxes) stays the same; coordinates and outputs may change between calls
    std::string topo;
    auto put = [&](const void* p, size_t nb) { topo.append(static_cast<const char*>(p), nb); };
    put(&n_sys, sizeof(n_sys));
    for (int b = 0; b < n_sys; ++b) {
      put(&sy[b].n_atoms, sizeof(sy[b].n_atoms));
      put(&sy[b].species, sizeof(sy[b].species));
      put(&sy[b].mask, sizeof(sy[b].mask));
      put(&sy[b].periodic, sizeof(sy[b].periodic));
      put(sy[b].box, sizeof(sy[b].box));
    }
    if (topo != h->list_sig) {
      h->lists_valid = false;
      h->list_sig = topo;
    }
    ++h->skin_calls;
  }
  // a call identical to the previous one (descriptors, sizes, arena) is replayed
  // from a CUDA graph: captured on its second occurrence, replayed afterwards
  if (!h->profile) {
    std::string sig;
    sig.reserve(64 + chunks.size() * sizeof(BatchParams));
    auto put = [&](const void* p, size_t nb) { sig.append(static_cast<const char*>(p), nb); };
    put(&n_sys, sizeof(n_sys));
    put(&n_in, sizeof(n_in));
    put(&h->arena, sizeof(h->arena));
    put(&ws.cap_r, sizeof(int));
    put(&ws.cap_a, sizeof(int));
    put(&ws.row_cap, sizeof(int));
    put(&ws.cell_cap, sizeof(int));
    const int skin_mode = ws.skin_state ? (h->lists_valid ? 1 : 2) : 0;
    put(&skin_mode, sizeof(skin_mode));
    put(&h->skin, sizeof(h->skin));
    put(&h->fused_chain, sizeof(h->fused_chain));
    put(&h->fused_aev_l1, sizeof(h->fused_aev_l1));
    put(&h->sparse_rows, sizeof(h->sparse_rows));
    put(&h->det, sizeof(h->det));
    // the kernels read only the first n_sys descriptors of a chunk
    for (const auto& bp : chunks)
      put(&bp, offsetof(BatchParams, sys) + (size_t)bp.n_sys * sizeof(SysIn));
    if (h->gexec && sig == h->gsig) {
      CU_TRY(cudaGraphLaunch(h->gexec, st));
      h->last_launches = h->last_launches_graph;
      h->last_n_in = n_in;
      h->lists_valid = true;
      return NNP_OK;
    }
    if (sig == h->last_sig) {
      if (!h->cap_stream) CU_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
      CU_TRY(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
      int launches = 0;
      rc = enqueue_batch(h, n_sys, sy, chunks, n_in, any_virial, h->cap_stream, &launches);
      cudaGraph_t graph = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &graph);
      if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      if (ec != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(NNP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
      }
      if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
      const cudaError_t ei = cudaGraphInstantiate(&h->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (ei != cudaSuccess) {
        h->gexec = nullptr;
        return fail(NNP_ERR_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(ei));
      }
      h->gsig = sig;
      h->last_launches_graph = launches;
      CU_TRY(cudaGraphLaunch(h->gexec, st));
      h->last_launches = launches;
      h->last_n_in = n_in;
      h->lists_valid = true;
      return NNP_OK;
    }
    h->last_sig = sig;
  }
  int launches = 0;
  rc = enqueue_batch(h, n_sys, sy, chunks, n_in, any_virial, st, &launches);
  if (rc) return rc;
  h->last_launches = launches;
  h->last_n_in = n_in;
  h->lists_valid = true;
  CU_TRY(cudaGetLastError());
  return NNP_OK;
}

int validate_system(const nnp_handle* h, const nnp_system_t& s) {
  if (s.n_atoms < 0) return fail(NNP_ERR_ARG, "negative atom count");
  if (!s.energy) return fail(NNP_ERR_ARG, "energy output pointer is null");
  if (s.n_atoms > 0 && (!s.coords || !s.species))
    return fail(NNP_ERR_ARG, "coords and species pointers are required");
  if (s.periodic) {
    const double rc = std::max(h->model->ac.rc_r, h->model->ac.rc_a);
    for (int c = 0; c < 3; ++c) {
      if (!std::isfinite(s.box[c]) || s.box[c] <= 0) return fail(NNP_ERR_ARG, "box edges must be positive");
      if (s.box[c] < 2 * rc)
        return fail(NNP_ERR_BOX_TOO_SMALL, "periodic box edge below twice the cutoff");
    }
  }
  return NNP_OK;
}

}  // namespace

// ================================================================ C ABI
extern "C" {

const char* nnp_last_error(void) { return g_err.c_str(); }

namespace {
bool alloc_host_words(nnp_handle* h) {
  void* p = nullptr;
  if (cudaMallocHost(&p, 16 + 10 * sizeof(double)) != cudaSuccess) return false;
  h->status_host = static_cast<int*>(p);
  h->out_host = reinterpret_cast<double*>(static_cast<char*>(p) + 16);
  return true;
}
}  // namespace

int nnp_create(const nnp_species_t* species, const nnp_aev_params_t* aev,
               const nnp_weights_t* weights, int precision, size_t hbm_budget_bytes,
               nnp_handle** out) {
  g_err.clear();
  if (!out) return fail(NNP_ERR_ARG, "null output handle");
  *out = nullptr;
  std::unique_ptr<Model> m(new Model);
  int rc = build_model(m.get(), species, aev, weights, precision);
  if (rc) return rc;
  nnp_handle* h = new nnp_handle;
  h->model = m.release();
  h->budget = hbm_budget_bytes;
  if (!alloc_host_words(h)) {
    nnp_destroy(h);
    return fail(NNP_ERR_CUDA, "cudaMallocHost failed");
  }
  *out = h;
  return NNP_OK;
}

int nnp_clone(const nnp_handle* src, nnp_handle** out) {
  if (!src || !out) return fail(NNP_ERR_ARG, "null argument");
  nnp_handle* h = new nnp_handle;
  h->model = src->model;
  h->model->refs.fetch_add(1);
  h->budget = src->budget;
  h->cap_r = src->cap_r;
  h->cap_a = src->cap_a;
  h->fused_chain = src->fused_chain;
  h->fused_aev_l1 = src->fused_aev_l1;
  h->det = src->det;
  if (!alloc_host_words(h)) {
    nnp_destroy(h);
    return fail(NNP_ERR_CUDA, "cudaMallocHost failed");
  }
  *out = h;
  return NNP_OK;
}

void nnp_destroy(nnp_handle* h) {
  if (!h) return;
  if (h->arena || h->stage || h->vjp_arena) cudaDeviceSynchronize();
  if (h->tc_state) mlp_tc_release(h->tc_state);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->arena) cudaFree(h->arena);
  if (h->stage) cudaFree(h->stage);
  if (h->vjp_arena) cudaFree(h->vjp_arena);
  if (h->status_host) cudaFreeHost(h->status_host);
  for (auto& pe : h->prof_pending) { cudaEventDestroy(pe.second.first); cudaEventDestroy(pe.second.second); }
  for (cudaEvent_t e : h->prof_pool) cudaEventDestroy(e);
  if (h->model && h->model->refs.fetch_sub(1) == 1) delete h->model;
  delete h;
}

int nnp_reserve(nnp_handle* h, int64_t max_atoms, int max_systems, int max_nr, int max_na) {
  g_err.clear();
  if (!h || max_atoms < 0 || max_systems < 0 || max_nr < 0 || max_na < 0)
    return fail(NNP_ERR_ARG, "bad argument");
  if (max_atoms > (1LL << 30)) return fail(NNP_ERR_ARG, "too many atoms");
  if (max_nr > kStageCap) return fail(NNP_ERR_UNSUPPORTED, "at most 512 radial neighbours per atom");
  if (max_nr) { h->cap_r = (int)align_up(max_nr, 32); h->dirty = true; }
  if (max_na) { h->cap_a = (int)align_up(std::min(max_na, h->cap_r), 32); h->dirty = true; }
  return ensure_arena(h, (int)std::max<int64_t>(max_atoms, h->cap_in), std::max(max_systems, h->cap_sys));
}

int nnp_energy_forces(nnp_handle* h, int64_t n_atoms, const float* coords, const uint8_t* species,
                      const double* box_host, const uint8_t* mask, double* energy, float* forces,
                      double* virial, void* stream) {
  g_err.clear();
  if (!h) return fail(NNP_ERR_ARG, "null handle");
  nnp_system_t s{};
  s.n_atoms = n_atoms;
  s.coords = coords;
  s.species = species;
  s.mask = mask;
  s.periodic = box_host != nullptr;
  if (box_host)
    for (int c = 0; c < 3; ++c) s.box[c] = box_host[c];
  s.energy = energy;
  s.forces = forces;
  s.virial = virial;
  int rc = validate_system(h, s);
  if (rc) return rc;
  return run_batch(h, 1, &s, static_cast<cudaStream_t>(stream));
}

int nnp_energy_forces_batch(nnp_handle* h, int n_sys, const nnp_system_t* systems, void* stream) {
  g_err.clear();
  if (!h || n_sys < 0 || (n_sys > 0 && !systems)) return fail(NNP_ERR_ARG, "bad argument");
  if (n_sys == 0) return NNP_OK;
  for (int b = 0; b < n_sys; ++b) {
    int rc = validate_system(h, systems[b]);
    if (rc) return rc;
  }
  return run_batch(h, n_sys, systems, static_cast<cudaStream_t>(stream));
}

namespace {

const char* bounds_site_name(int site) {
  static const char* names[kSiteCount] = {
      "an unknown site", "cell binning (cell index)", "scatter (packed position)",
      "neighbour search (list entry)", "AEV kernels (staged neighbour)", "AEV forward (row slot)",
      "AEV backward (force target)", "AEV backward (triplet slot)",
      "AEV backward (dense-centre list)", "finalize (row slot)",
      "tensor-core epilogue (output row)"};
  return (site > 0 && site < kSiteCount) ? names[site] : names[0];
}

// enqueue the read-back and reset of the device status word on st
cudaError_t enqueue_status_read(nnp_handle* h, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(h->status_host, h->ws.status, 4 * sizeof(int),
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->ws.status, 0, 4 * sizeof(int), st);
  return e;
}

// the outcome of the status word read back by enqueue_status_read (after a sync)
int status_result(nnp_handle* h) {
  const int f = h->status_host[0];
  if (f & kStSpecies) return fail(NNP_ERR_SPECIES, "species index out of range");
  if (f & kStNonFinite) return fail(NNP_ERR_NONFINITE, "non-finite coordinate in the ML region");
  if (f & kStTimeout) return fail(NNP_ERR_TIMEOUT, "a bounded device wait gave up");
  if (f & kStBounds)
    return fail(NNP_ERR_BOUNDS, std::string("index out of range at ") +
                                    bounds_site_name(h->status_host[3]) + " (access skipped)");
  if (f & (kStCapacity | kStCells)) {
    const int need_r = h->status_host[1], need_a = h->status_host[2];
    if (need_r > kStageCap)
      return fail(NNP_ERR_UNSUPPORTED, "more than 512 neighbours inside the radial cutoff");
    h->cap_r = std::max(h->cap_r, (int)align_up(need_r + need_r / 8 + 1, 32));
    h->cap_r = std::min(h->cap_r, kStageCap);
    h->cap_a = std::max(h->cap_a, (int)align_up(need_a + need_a / 8 + 1, 32));
    h->cap_a = std::min(h->cap_a, h->cap_r);
    h->dirty = true;
    return fail(NNP_ERR_CAPACITY, "neighbour list over capacity (grown to " +
                                      std::to_string(h->cap_r) + " / " + std::to_string(h->cap_a) +
                                      "); repeat the call");
  }
  return NNP_OK;
}

}  // namespace

int nnp_sync_status(nnp_handle* h, void* stream) {
  g_err.clear();
  if (!h) return fail(NNP_ERR_ARG, "null handle");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (h->arena) CU_TRY(enqueue_status_read(h, st));
  CU_TRY(cudaStreamSynchronize(st));
  return h->arena ? status_result(h) : NNP_OK;
}

int nnp_energy_forces_host(nnp_handle* h, int64_t n, const float* coords_h,
                           const uint8_t* species_h, const double* box_host, const uint8_t* mask_h,
                           double* energy_h, float* forces_h, double* virial_h) {
  g_err.clear();
  if (!h || n < 0 || !energy_h || (n > 0 && (!coords_h || !species_h || !forces_h)))
    return fail(NNP_ERR_ARG, "bad argument");
  // staging: coords, forces, species, mask, energy, virial
  const size_t b_xyz = align_up((size_t)n * 12, 256), b_sp = align_up((size_t)n, 256);
  const size_t need = 2 * b_xyz + 2 * b_sp + 256 + 256;
  if (need > h->stage_bytes) {
    if (h->stage) { CU_TRY(cudaDeviceSynchronize()); cudaFree(h->stage); h->stage = nullptr; }
    CU_TRY(cudaMalloc(&h->stage, need));
    h->stage_bytes = need;
  }
  char* base = static_cast<char*>(h->stage);
  float* d_xyz = reinterpret_cast<float*>(base);
  float* d_f = reinterpret_cast<float*>(base + b_xyz);
  uint8_t* d_sp = reinterpret_cast<uint8_t*>(base + 2 * b_xyz);
  uint8_t* d_mask = reinterpret_cast<uint8_t*>(base + 2 * b_xyz + b_sp);
  double* d_e = reinterpret_cast<double*>(base + 2 * b_xyz + 2 * b_sp);
  double* d_v = reinterpret_cast<double*>(base + 2 * b_xyz + 2 * b_sp + 256);
  cudaStream_t st = nullptr;
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (n > 0) {
      CU_TRY(cudaMemcpyAsync(d_xyz, coords_h, (size_t)n * 12, cudaMemcpyHostToDevice, st));
      CU_TRY(cudaMemcpyAsync(d_sp, species_h, (size_t)n, cudaMemcpyHostToDevice, st));
      if (mask_h) CU_TRY(cudaMemcpyAsync(d_mask, mask_h, (size_t)n, cudaMemcpyHostToDevice, st));
    }
    int rc = nnp_energy_forces(h, n, d_xyz, d_sp, box_host, mask_h ? d_mask : nullptr, d_e, d_f,
                               virial_h ? d_v : nullptr, st);
    if (rc) return rc;
    // energy and virial land in pinned words and the status read joins the same
    // stream, so that the call synchronises once
    CU_TRY(cudaMemcpyAsync(h->out_host, d_e, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (n > 0) CU_TRY(cudaMemcpyAsync(forces_h, d_f, (size_t)n * 12, cudaMemcpyDeviceToHost, st));
    if (virial_h)
      CU_TRY(cudaMemcpyAsync(h->out_host + 1, d_v, 9 * sizeof(double), cudaMemcpyDeviceToHost, st));
    rc = nnp_sync_status(h, st);
    if (rc == NNP_OK) {
      *energy_h = h->out_host[0];
      if (virial_h) std::memcpy(virial_h, h->out_host + 1, 9 * sizeof(double));
    }
    if (rc != NNP_ERR_CAPACITY) return rc;
  }
  return fail(NNP_ERR_CAPACITY, "neighbour list over capacity after one retry");
}

// ---------------------------------------------------------------- force VJP
namespace {

size_t carve_vjp(nnp_handle* h, char* base, int rows, int n) {
  const Model& m = *h->model;
  const int E = m.md.E, Dp = m.ac.Dp;
  const size_t w1 = (size_t)rows * E * m.md.h1, w2 = (size_t)rows * E * m.md.h2, w3 = (size_t)rows * E * m.md.h3;
  Carve c{base};
  VjpBufs& v = h->vb;
  v.v_pos = c.take<float4>(n);
  v.df_pos = c.take<float4>(n);
  v.gE_row = c.take<float>(rows);
  v.U = c.take<float>((size_t)rows * Dp);
  v.Q = c.take<float>((size_t)rows * Dp);
  float** l1[] = {&v.H1, &v.D1, &v.Z1d, &v.H1d, &v.A1h, &v.A1z, &v.dl1, &v.dl1d};
  for (float** q : l1) *q = c.take<float>(w1);
  float** l2[] = {&v.H2, &v.D2, &v.Z2d, &v.H2d, &v.A2h, &v.A2z, &v.dl2, &v.dl2d};
  for (float** q : l2) *q = c.take<float>(w2);
  float** l3[] = {&v.H3, &v.D3, &v.Z3d, &v.H3d, &v.dl3, &v.dl3d};
  for (float** q : l3) *q = c.take<float>(w3);
  v.e_row = c.take<float>((size_t)E * rows);
  return align_up(c.off, 256);
}

int ensure_vjp(nnp_handle* h) {
  const int rows = h->ws.row_cap, n = std::max(h->cap_in, 1);
  if (h->vjp_arena && rows <= h->vjp_rows) {
    // neighbour capacities may have grown since the buffers were made
    CU_TRY(vjp_set_smem(h->ws));
    return NNP_OK;
  }
  const size_t bytes = carve_vjp(h, nullptr, rows, n);
  if (h->vjp_arena) {
    CU_TRY(cudaDeviceSynchronize());
    cudaFree(h->vjp_arena);
    h->vjp_arena = nullptr;
  }
  if (cudaMalloc(&h->vjp_arena, bytes) != cudaSuccess) {
    cudaGetLastError();
    h->vjp_arena = nullptr;
    h->vjp_rows = 0;
    return fail(NNP_ERR_OOM, "cudaMalloc of the force-VJP buffers failed");
  }
  CU_TRY(cudaMemset(h->vjp_arena, 0, bytes));
  h->vjp_bytes = bytes;
  h->vjp_rows = rows;
  carve_vjp(h, static_cast<char*>(h->vjp_arena), rows, n);
  CU_TRY(vjp_set_smem(h->ws));
  return NNP_OK;
}

GemmArgs gemm_base(const Ws& ws, const Model& m) {
  GemmArgs g{};
  g.alpha = m.alpha;
  g.seg_start = ws.seg_start;
  g.S = m.md.S;
  return g;
}

// forward, tangent forward and forward-over-reverse of the networks (FP32)
void vjp_networks(nnp_handle* h, cudaStream_t st) {
  const Model& m = *h->model;
  const Ws& ws = h->ws;
  const VjpBufs& v = h->vb;
  const MlpWeights& w = m.mw;
  const int E = m.md.E, S = m.md.S, Dp = m.ac.Dp, h1 = m.md.h1, h2 = m.md.h2, h3 = m.md.h3;
  const int R = ws.row_cap;
  auto L1 = [&](const float* A, int epi, float* out, float* out2, const float* aux) {
    GemmArgs g = gemm_base(ws, m);
    g.A = A; g.lda = Dp; g.a_net = 0;
    g.B = w.W1cat; g.b_s = (long long)E * h1 * Dp; g.b_e = 0; g.ldb = Dp;
    g.bias = w.b1cat; g.bias_s = (long long)E * h1; g.bias_e = 0;
    g.N = E * h1; g.K = Dp;
    g.out = out; g.out2 = out2; g.ldo = E * h1; g.out_net = 0;
    g.aux = aux; g.ld_aux = E * h1; g.aux_net = 0;
    g.epi = epi;
    launch_gemm_fp32(g, R, st, 1);
  };
  // per-member layer: out[:, e*n_out] = A[:, e*k] B_{e,s}^T
  auto Lm = [&](const float* A, int k, const float* B, int n_out, const float* bias, int epi, float* out,
                float* out2, const float* aux) {
    GemmArgs g = gemm_base(ws, m);
    g.A = A; g.lda = E * k; g.a_net = k;
    g.B = B; g.b_s = (long long)n_out * k; g.b_e = (long long)S * n_out * k; g.ldb = k;
    g.bias = bias; g.bias_s = n_out; g.bias_e = (long long)S * n_out;
    g.N = n_out; g.K = k;
    g.out = out; g.out2 = out2; g.ldo = E * n_out; g.out_net = n_out;
    g.aux = aux; g.ld_aux = E * n_out; g.aux_net = n_out;
    g.epi = epi;
    launch_gemm_fp32(g, R, st, E);
  };
  L1(ws.aev, kEpiCelu, v.H1, v.D1, nullptr);
  Lm(v.H1, h1, w.W2, h2, w.b2, kEpiCelu, v.H2, v.D2, nullptr);
  Lm(v.H2, h2, w.W3, h3, w.b3, kEpiCelu, v.H3, v.D3, nullptr);
  L1(v.U, kEpiStoreMul, v.Z1d, v.H1d, v.D1);
  Lm(v.H1d, h1, w.W2, h2, nullptr, kEpiStoreMul, v.Z2d, v.H2d, v.D2);
  Lm(v.H2d, h2, w.W3, h3, nullptr, kEpiStoreMul, v.Z3d, v.H3d, v.D3);
  launch_vjp_out3(ws, v, w.w4, S, E, h3, m.alpha, st);
  Lm(v.dl3, h3, w.W3T, h2, nullptr, kEpiStore, v.A2h, nullptr, nullptr);
  Lm(v.dl3d, h3, w.W3T, h2, nullptr, kEpiStore, v.A2z, nullptr, nullptr);
  launch_vjp_delta(ws, S, E * h2, v.A2h, v.A2z, v.D2, v.Z2d, v.dl2, v.dl2d, m.alpha, st);
  Lm(v.dl2, h2, w.W2T, h1, nullptr, kEpiStore, v.A1h, nullptr, nullptr);
  Lm(v.dl2d, h2, w.W2T, h1, nullptr, kEpiStore, v.A1z, nullptr, nullptr);
  launch_vjp_delta(ws, S, E * h1, v.A1h, v.A1z, v.D1, v.Z1d, v.dl1, v.dl1d, m.alpha, st);
  auto B1 = [&](const float* A, float* out) {
    GemmArgs g = gemm_base(ws, m);
    g.A = A; g.lda = E * h1; g.a_net = 0;
    g.B = w.W1Tcat; g.b_s = (long long)Dp * E * h1; g.b_e = 0; g.ldb = E * h1;
    g.N = Dp; g.K = E * h1;
    g.out = out; g.ldo = Dp; g.out_net = 0;
    g.epi = kEpiStore;
    launch_gemm_fp32(g, R, st, 1);
  };
  B1(v.dl1, ws.dEdG);
  B1(v.dl1d, v.Q);
}

void vjp_weight_grads(nnp_handle* h, float* out, cudaStream_t st) {
  const Model& m = *h->model;
  const Ws& ws = h->ws;
  const VjpBufs& v = h->vb;
  const int E = m.md.E, S = m.md.S, D = m.ac.D, Dp = m.ac.Dp, h1 = m.md.h1, h2 = m.md.h2, h3 = m.md.h3;
  const long long off2 = (long long)h1 * D + h1, off3 = off2 + (long long)h2 * h1 + h2;
  const long long off4 = off3 + (long long)h3 * h2 + h3;
  const long long per_net = off4 + h3 + 1;
  WgradArgs a{};
  a.S = S; a.scale = 1.f / E; a.out = out; a.per_net = per_net;
  a.X1 = v.dl1; a.X2 = v.dl1d; a.ldx = E * h1; a.x_net = h1;
  a.Y1 = ws.aev; a.Y2 = v.U; a.ldy = Dp; a.y_net = 0;
  a.n_out = h1; a.n_in = Dp; a.n_in_real = D; a.layer_off = 0;
  a.feat_of_col = m.feat_of_col_dev;   // W1's columns back in the paper's feature order
  launch_wgrad(a, ws, v, E, st);
  a.feat_of_col = nullptr;
  a.X1 = v.dl2; a.X2 = v.dl2d; a.ldx = E * h2; a.x_net = h2;
  a.Y1 = v.H1; a.Y2 = v.H1d; a.ldy = E * h1; a.y_net = h1;
  a.n_out = h2; a.n_in = h1; a.n_in_real = h1; a.layer_off = off2;
  launch_wgrad(a, ws, v, E, st);
  a.X1 = v.dl3; a.X2 = v.dl3d; a.ldx = E * h3; a.x_net = h3;
  a.Y1 = v.H2; a.Y2 = v.H2d; a.ldy = E * h2; a.y_net = h2;
  a.n_out = h3; a.n_in = h2; a.n_in_real = h2; a.layer_off = off3;
  launch_wgrad(a, ws, v, E, st);
  launch_wgrad_out(ws, v, S, E, h3, out, per_net, off4, st);
}

}  // namespace

extern "C" int nnp_force_vjp_batch(nnp_handle* h, int n_sys, const nnp_vjp_system_t* vs,
                                   float* dL_dweights, void* stream) {
  g_err.clear();
  if (!h || n_sys < 1 || !vs || !dL_dweights) return fail(NNP_ERR_ARG, "bad argument");
  const Model& m = *h->model;
  if (m.net == kNetBf16) return fail(NNP_ERR_UNSUPPORTED, "the force VJP runs FP32 handles");
  std::vector<nnp_system_t> sy(n_sys);
  long long n_in_ll = 0;
  for (int b = 0; b < n_sys; ++b) {
    sy[b] = vs[b].sys;
    int rc = validate_system(h, sy[b]);
    if (rc) return rc;
    if (sy[b].n_atoms > 0 && (!vs[b].dL_dF || !vs[b].dL_dcoords))
      return fail(NNP_ERR_ARG, "dL_dF and dL_dcoords are required");
    if (sy[b].n_atoms == 0) return fail(NNP_ERR_ARG, "empty system in a force VJP batch");
    n_in_ll += sy[b].n_atoms;
  }
  if (n_in_ll > (1LL << 30)) return fail(NNP_ERR_ARG, "too many atoms in one call");
  const int n_in = (int)n_in_ll;
  int rc = ensure_arena(h, n_in, n_sys);
  if (rc) return rc;
  if ((rc = ensure_vjp(h))) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->ws.n_sys = n_sys;
  h->ws.n_in = n_in;
  // the VJP's FP32 network chain reads the FP32 AEV rows (a split handle's
  // energy calls write only the two BF16 planes)
  Ws ws = h->ws;
  ws.aev_h = nullptr;
  ws.aev_l = nullptr;
  ws.row_mask = nullptr;      // the FP32 chain reads whole rows
  ws.tile_mask = nullptr;
  // the deterministic mode covers energy and force calls, not the VJP (whose
  // dual backward adds atomically): the forces here add atomically as well
  ws.fr_det = ws.fa_det = ws.fs_det = nullptr;
  ws.e_det = ws.v_det = nullptr;
  h->last_aev_fp32 = true;
  h->last_sparse = false;
  // the force VJP builds its own lists at the cutoffs in the shared buffers:
  // persistent lists of energy calls are rebuilt on the next such call
  struct SkinOff {
    Ws& w;
    int* saved;
    explicit SkinOff(Ws& w_) : w(w_), saved(w_.skin_state) { w.skin_state = nullptr; }
    ~SkinOff() { w.skin_state = saved; }
  } skin_off(ws);
  h->lists_valid = false;
  int in_base = 0;
  std::vector<BatchParams> chunks;
  for (int b0 = 0; b0 < n_sys; b0 += kMaxBatchParam) {
    BatchParams bp{};
    bp.sys_base = b0;
    bp.n_sys = std::min(kMaxBatchParam, n_sys - b0);
    for (int k = 0; k < bp.n_sys; ++k) {
      const nnp_system_t& s = sy[b0 + k];
      SysIn& si = bp.sys[k];
      si.coords = s.coords; si.species = s.species; si.mask = s.mask;
      si.energy = s.energy; si.forces = s.forces; si.virial = nullptr; si.atom_e = s.atom_energies;
      si.n_in = (int)s.n_atoms; si.in_base = in_base; si.periodic = s.periodic ? 1 : 0;
      for (int c = 0; c < 3; ++c) split_box(s.periodic ? s.box[c] : 1.0, &si.box_hi[c], &si.box_lo[c], &si.inv_box[c]);
      si.dLdF = vs[b0 + k].dL_dF;
      si.dLdR = vs[b0 + k].dL_dcoords;
      si.gE = vs[b0 + k].dL_dE;
      in_base += (int)s.n_atoms;
    }
    chunks.push_back(bp);
  }
  for (const auto& bp : chunks) launch_init_chunk(ws, bp, st);
  for (const auto& bp : chunks) {
    int n_chunk = 0;
    for (int k = 0; k < bp.n_sys; ++k) n_chunk += bp.sys[k].n_in;
    launch_prep_atoms(ws, bp, n_chunk, m.ac.S, st);
  }
  launch_setup(ws, m.ac, st);
  launch_bin(ws, n_in, st);
  launch_scan(ws, st);
  launch_scatter(ws, n_in, st);
  launch_neighbors(ws, n_in, m.ac, st);
  launch_aev_fwd(ws, n_in, m.ac, st);
  launch_vjp_zero(ws, h->vb, n_in, st);
  launch_gather_v(ws, h->vb, n_in, st);
  launch_aev_jvp(ws, m.ac, h->vb, n_in, st);
  vjp_networks(h, st);
  launch_aev_bwd(ws, n_in, m.ac, 0, st);
  launch_aev_bwd_dual(ws, m.ac, h->vb, n_in, st);
  launch_finalize_e(ws, n_in, h->vb.e_row, m.md.E, ws.row_cap, m.ebias, st);
  launch_vjp_scatter(ws, h->vb, n_in, st);
  vjp_weight_grads(h, dL_dweights, st);
  h->last_n_in = n_in;
  CU_TRY(cudaGetLastError());
  return NNP_OK;
}

extern "C" int nnp_force_vjp(nnp_handle* h, int64_t n_atoms, const float* coords, const uint8_t* species,
                             const double* box_host, const uint8_t* mask, double dL_dE, const float* dL_dF,
                             double* energy, float* forces, float* dL_dcoords, float* dL_dweights,
                             void* stream) {
  nnp_vjp_system_t v{};
  v.sys.n_atoms = n_atoms;
  v.sys.coords = coords;
  v.sys.species = species;
  v.sys.mask = mask;
  v.sys.periodic = box_host != nullptr;
  if (box_host)
    for (int c = 0; c < 3; ++c) v.sys.box[c] = box_host[c];
  v.sys.energy = energy;
  v.sys.forces = forces;
  v.dL_dE = dL_dE;
  v.dL_dF = dL_dF;
  v.dL_dcoords = dL_dcoords;
  return nnp_force_vjp_batch(h, 1, &v, dL_dweights, stream);
}

extern "C" int64_t nnp_n_weights(const nnp_handle* h) {
  if (!h) return -1;
  const Model& m = *h->model;
  const long long D = m.ac.D, h1 = m.md.h1, h2 = m.md.h2, h3 = m.md.h3;
  const long long per = h1 * D + h1 + h2 * h1 + h2 + h3 * h2 + h3 + h3 + 1;
  return per * m.md.S * m.md.E;
}

int nnp_aev_dim(const nnp_handle* h) { return h ? h->model->ac.D : -1; }

int nnp_build_flags(void) { return kBoundsChecked ? NNP_BUILD_BOUNDS_CHECKS : 0; }

int nnp_debug_check_index(int site, int64_t i, int64_t n, int* status) {
  g_err.clear();
  if (!status || site <= kSiteNone || site >= kSiteCount) {
    fail(NNP_ERR_ARG, "bad argument");
    return -1;
  }
  return bounds_ok(status, site, i, n) ? 1 : 0;
}
int nnp_debug_tile_masks(nnp_handle* h, void* stream, uint32_t* out_host, int max_tiles,
                         int* n_tiles) {
  g_err.clear();
  if (!h || !out_host || !n_tiles || max_tiles < 0) return fail(NNP_ERR_ARG, "bad argument");
  *n_tiles = 0;
  if (!h->arena || !h->last_sparse) return NNP_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CU_TRY(cudaStreamSynchronize(st));
  int seg = 0;
  CU_TRY(cudaMemcpy(&seg, h->ws.seg_start + h->model->ac.S, sizeof(int), cudaMemcpyDeviceToHost));
  const int n = std::min(seg / kRowTile, max_tiles);
  if (n > 0) CU_TRY(cudaMemcpy(out_host, h->ws.tile_mask, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  *n_tiles = n;
  return NNP_OK;
}

int nnp_set_deterministic(nnp_handle* h, int enable) {
  g_err.clear();
  if (!h) return fail(NNP_ERR_ARG, "null handle");
  if (h->det != (enable != 0)) {
    h->det = enable != 0;
    h->dirty = true;   // the arena gains or drops the per-contribution buffers
    h->lists_valid = false;
  }
  return NNP_OK;
}

int nnp_set_sparse_rows(nnp_handle* h, int enable) {
  g_err.clear();
  if (!h) return fail(NNP_ERR_ARG, "null handle");
  h->sparse_rows = enable != 0;
  return NNP_OK;
}

int nnp_set_fused_aev_l1(nnp_handle* h, int enable) {
  g_err.clear();
  if (!h) return fail(NNP_ERR_ARG, "null handle");
  h->fused_aev_l1 = enable != 0;
  return NNP_OK;
}

int nnp_set_fused_chain(nnp_handle* h, int enable) {
  g_err.clear();
  if (!h) return fail(NNP_ERR_ARG, "null handle");
  h->fused_chain = enable != 0;
  mlp_tc_use_chain(h->tc_state, h->fused_chain);
  return NNP_OK;
}

int nnp_network_path(const nnp_handle* h) {
  if (!h) return -1;
  const int net = h->model->net;
  return net == kNetBf16 ? NNP_BF16_MLP : net == kNetSplit ? NNP_FP32_SPLIT : NNP_FP32_SIMT;
}
int nnp_last_launch_count(const nnp_handle* h) { return h ? h->last_launches : -1; }

int nnp_set_skin(nnp_handle* h, float skin) {
  g_err.clear();
  if (!h) return fail(NNP_ERR_ARG, "null handle");
  if (!(skin >= 0.f) || skin > 3.f) return fail(NNP_ERR_ARG, "skin must be in [0, 3] A");
  if (skin != h->skin) {
    h->skin = skin;
    h->dirty = true;          // the arena gains or drops the reference coordinates
    h->lists_valid = false;
  }
  return NNP_OK;
}

int nnp_list_stats(nnp_handle* h, void* stream, int64_t* builds, int64_t* calls) {
  g_err.clear();
  if (!h || !builds || !calls) return fail(NNP_ERR_ARG, "null argument");
  *builds = 0;
  *calls = h->skin_calls;
  if (!h->arena || !h->ws.skin_state) return NNP_OK;
  CU_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  int st[4];
  CU_TRY(cudaMemcpy(st, h->ws.skin_state, sizeof(st), cudaMemcpyDeviceToHost));
  *builds = st[2];
  return NNP_OK;
}

int nnp_debug_wait_probe(nnp_handle* h, unsigned limit, void* stream) {
  g_err.clear();
  if (!h) return fail(NNP_ERR_ARG, "null handle");
  if (!h->arena) {
    int rc = ensure_arena(h, 1, 1);
    if (rc) return rc;
  }
  launch_wait_probe(h->ws.status, limit, static_cast<cudaStream_t>(stream));
  CU_TRY(cudaGetLastError());
  return NNP_OK;
}

int nnp_profile(nnp_handle* h, int enable) {
  if (!h) return fail(NNP_ERR_ARG, "null handle");
  h->profile = enable != 0;
  return NNP_OK;
}

int nnp_profile_read(nnp_handle* h, int reset, double* ms_out, long long* calls_out,
                     int max_stages, int* n_stages) {
  if (!h) return fail(NNP_ERR_ARG, "null handle");
  for (auto& pe : h->prof_pending) {
    CU_TRY(cudaEventSynchronize(pe.second.second));
    float ms = 0.f;
    CU_TRY(cudaEventElapsedTime(&ms, pe.second.first, pe.second.second));
    h->prof_ms[pe.first] += ms;
    h->prof_calls[pe.first] += 1;
    h->prof_pool.push_back(pe.second.first);
    h->prof_pool.push_back(pe.second.second);
  }
  h->prof_pending.clear();
  const int n = std::min(max_stages, kNumStages);
  for (int i = 0; i < n; ++i) {
    if (ms_out) ms_out[i] = h->prof_ms[i];
    if (calls_out) calls_out[i] = h->prof_calls[i];
  }
  if (n_stages) *n_stages = kNumStages;
  if (reset)
    for (int i = 0; i < kNumStages; ++i) { h->prof_ms[i] = 0; h->prof_calls[i] = 0; }
  return NNP_OK;
}

const char* nnp_profile_stage_name(int i) {
  return (i >= 0 && i < kNumStages) ? kStageNames[i] : "";
}

// ---------------------------------------------------------------- diagnostics
// Rows of the last call in batch input-atom order: which = 0 AEV (on the BF16
// path its BF16 copy, widened), 1 dE/dG.
// out: device float [n_in_total, D]; rows of atoms outside the mask untouched.
int nnp_debug_rows(nnp_handle* h, int which, float* out, void* stream) {
  if (!h || !h->arena || !out) return fail(NNP_ERR_ARG, "bad argument");
  if (which == 0 && !h->last_aev_stored)
    return fail(NNP_ERR_UNSUPPORTED, "the last call fed the AEV to the first layer on chip; no AEV rows were stored");
  const bool planes = which == 0 && !h->last_aev_fp32;
  const float* src = which == 0 ? h->ws.aev : h->ws.dEdG;
  const uint16_t* src_h = planes ? h->ws.aev_h : nullptr;
  const uint16_t* src_l = planes ? h->ws.aev_l : nullptr;
  Ws gw = h->ws;
  if (!h->last_sparse) gw.row_mask = nullptr;   // the last call wrote whole rows
  launch_gather_rows(gw, h->last_n_in, src, src_h, src_l, h->model->ac.Dp, h->model->ac.D,
                     h->model->col_of_feat_dev, out, which == 1, static_cast<cudaStream_t>(stream));
  CU_TRY(cudaGetLastError());
  return NNP_OK;
}

int nnp_debug_cell_grid(const float* len, float rc, int64_t n_atoms, int* nc_out,
                        int64_t* cells_out) {
  g_err.clear();
  if (!len || !nc_out || !cells_out || !(rc > 0.f) || n_atoms < 0)
    return fail(NNP_ERR_ARG, "bad argument");
  const float l[3] = {len[0], len[1], len[2]};
  *cells_out = cell_grid(l, rc, 2 * (long long)n_atoms + 27, nc_out);
  return NNP_OK;
}

// Neighbour lists of the last call in input-atom order: out[i][t] = input index
// of the t-th neighbour of atom i (radial list, or angular if angular != 0),
// -1 past the end.  out: device int32 [n_in_total, cap].
int nnp_debug_neighbors(nnp_handle* h, int angular, int cap, int* out, void* stream) {
  if (!h || !h->arena || !out || cap <= 0) return fail(NNP_ERR_ARG, "bad argument");
  launch_gather_nbrs(h->ws, h->last_n_in, angular, cap, out, static_cast<cudaStream_t>(stream));
  CU_TRY(cudaGetLastError());
  return NNP_OK;
}

}  // extern "C"

// ================================================================ allocation-free variant
// nnp_energy_forces_noalloc: the nnp_energy_forces kernel chain with its work
// buffers carved from one file-scope device array instead of the handle's
// cudaMalloc'd arena.  For callers that may not have the library allocate
// device memory while they run (an engine that owns the whole HBM budget, or a
// time loop where an allocation would stall or fail).  Nothing here allocates:
// the array is part of the loaded module, and its device address is looked up
// once per device.
namespace {

constexpr size_t kNoAllocBytes = NNP_NOALLOC_SCRATCH_BYTES;
constexpr int kNoAllocCapR = 256;  // radial neighbours per atom held by the fixed lists
constexpr int kNoAllocCapA = 96;   // angular neighbours per atom
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_base[kNoAllocMaxDevices] = {nullptr};

// device address of the scratch array on the current device (looked up on first use)
int noalloc_base(void** out) {
  int dev = -1;
  CU_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(NNP_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_base[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(NNP_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array: ") +
                                    cudaGetErrorString(e));
    g_noalloc_base[dev] = p;
  }
  *out = g_noalloc_base[dev];
  return NNP_OK;
}

// lay out the buffers of one n-atom system over `base` (nullptr: only measure)
size_t noalloc_carve(const Model& m, int n_atoms, char* base, Ws* ws, MlpBufs* mb) {
  const int S = m.ac.S, Dp = m.ac.Dp, E = m.md.E;
  const size_t n = std::max(n_atoms, 1);
  const size_t cells = 2 * n + 27;
  const size_t rows = n + (size_t)S * kRowTile;
  Carve c{base};
  ws->status = c.take<int>(4);
  ws->sys = c.take<SysDev>(1);
  ws->n_sys = 1;
  ws->n_in = n_atoms;
  ws->cell_cap = (int)cells;
  ws->row_cap = (int)rows;
  ws->cap_r = kNoAllocCapR;
  ws->cap_a = kNoAllocCapA;
  ws->species_count = c.take<int>(kMaxSpecies);
  ws->species_fill = c.take<int>(kMaxSpecies);
  ws->seg_start = c.take<int>(kMaxSpecies + 1);
  ws->totals = c.take<int>(8);
  ws->cell_count = c.take<int>(cells);
  ws->cell_start = c.take<int>(cells + 1);
  ws->in_cell = c.take<int>(n);
  ws->in_rank = c.take<int>(n);
  ws->in_slot = c.take<int>(n);
  ws->in_sys = c.take<int>(n);
  ws->xyzq = c.take<float4>(n);
  ws->pos_src = c.take<int>(n);
  ws->pos_slot = c.take<int>(n);
  ws->pos_sys = c.take<int>(n);
  ws->pos_cell = c.take<int>(n);
  ws->slot_pos = nullptr;
  ws->row_mask = nullptr;
  ws->tile_mask = nullptr;
  ws->nb_cnt = c.take<uint16_t>(n * 16);
  ws->nb_r = c.take<int>(n * kNoAllocCapR);
  ws->nb_a = c.take<int>(n * kNoAllocCapA);
  ws->aev = c.take<float>(rows * Dp);
  ws->dEdG = c.take<float>(rows * Dp);
  ws->atom_e = c.take<float>(rows);
  ws->f_pos = c.take<float4>(n);
  ws->heavy = c.take<int>(n);
  ws->fr_det = ws->fa_det = ws->fs_det = nullptr;
  ws->e_det = ws->v_det = nullptr;
  *mb = MlpBufs{};
  if (!mlp_fused_supported(m.md)) {   // the fused kernel needs no activation buffers
    mb->H1 = c.take<float>(rows * E * m.md.h1);
    mb->D1 = c.take<float>(rows * E * m.md.h1);
    mb->H2 = c.take<float>(rows * E * m.md.h2);
    mb->D2 = c.take<float>(rows * E * m.md.h2);
    mb->d3 = c.take<float>(rows * E * m.md.h3);
  }
  mb->e_row = c.take<float>((size_t)E * rows);
  mb->aev_h = nullptr;
  ws->aev_h = nullptr;
  return align_up(c.off, 256);
}

}  // namespace

extern "C" int nnp_energy_forces_noalloc(nnp_handle* h, int64_t n_atoms, const float* coords,
                                         const uint8_t* species, const double* box_host,
                                         const uint8_t* mask, double* energy, float* forces,
                                         double* virial, void* stream) {
  g_err.clear();
  if (!h) return fail(NNP_ERR_ARG, "null handle");
  const Model& m = *h->model;
  if (m.net == kNetBf16)
    return fail(NNP_ERR_UNSUPPORTED, "the allocation-free entry point runs FP32 handles only");
  nnp_system_t s{};
  s.n_atoms = n_atoms;
  s.coords = coords;
  s.species = species;
  s.mask = mask;
  s.periodic = box_host != nullptr;
  if (box_host)
    for (int c = 0; c < 3; ++c) s.box[c] = box_host[c];
  s.energy = energy;
  s.forces = forces;
  s.virial = virial;
  int rc = validate_system(h, s);
  if (rc) return rc;
  if (n_atoms > (1 << 24)) return fail(NNP_ERR_ARG, "too many atoms");
  Ws ws{};
  MlpBufs mb{};
  const size_t need = noalloc_carve(m, (int)n_atoms, nullptr, &ws, &mb);
  if (need > kNoAllocBytes)
    return fail(NNP_ERR_ARG, "system needs " + std::to_string(need) +
                                 " bytes of work space; the allocation-free entry point has " +
                                 std::to_string(kNoAllocBytes) + " (NNP_NOALLOC_SCRATCH_BYTES)");
  void* base = nullptr;
  rc = noalloc_base(&base);
  if (rc) return rc;
  noalloc_carve(m, (int)n_atoms, static_cast<char*>(base), &ws, &mb);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaGetLastError();  // a stale error of an earlier runtime call is not this call's
  // the fixed neighbour lists may need more shared memory than other handles set up
  CU_TRY(aev_ensure_smem(ws));
  CU_TRY(mlp_fused_ensure_smem(m.md));
  // the status word starts at zero on every call; the kernels clear the rest
  CU_TRY(cudaMemsetAsync(ws.status, 0, 4 * sizeof(int), st));
  if (n_atoms == 0) {
    CU_TRY(cudaMemsetAsync(energy, 0, sizeof(double), st));
    if (virial) CU_TRY(cudaMemsetAsync(virial, 0, 9 * sizeof(double), st));
  } else {
    BatchParams bp{};
    bp.sys_base = 0;
    bp.n_sys = 1;
    SysIn& si = bp.sys[0];
    si.coords = coords;
    si.species = species;
    si.mask = mask;
    si.energy = energy;
    si.forces = forces;
    si.virial = virial;
    si.atom_e = nullptr;
    si.n_in = (int)n_atoms;
    si.in_base = 0;
    si.periodic = s.periodic;
    for (int c = 0; c < 3; ++c)
      split_box(s.periodic ? s.box[c] : 1.0, &si.box_hi[c], &si.box_lo[c], &si.inv_box[c]);
    const int n = (int)n_atoms;
    // each stage's launch status is checked so that a failure names its stage
    auto stage_ok = [&](const char* name) -> int {
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return fail(NNP_ERR_CUDA, std::string(name) + ": " + cudaGetErrorString(e));
      return NNP_OK;
    };
    launch_init_chunk(ws, bp, st);
    if ((rc = stage_ok("init"))) return rc;
    launch_prep_atoms(ws, bp, n, m.ac.S, st);
    if ((rc = stage_ok("prep"))) return rc;
    launch_setup(ws, m.ac, st);
    launch_bin(ws, n, st);
    launch_scan(ws, st);
    launch_scatter(ws, n, st);
    if ((rc = stage_ok("cells"))) return rc;
    launch_neighbors(ws, n, m.ac, st);
    if ((rc = stage_ok("neighbors"))) return rc;
    launch_aev_fwd(ws, n, m.ac, st);
    if ((rc = stage_ok("aev_fwd"))) return rc;
    launch_mlp_fp32(ws, m.md, m.mw, mb, m.alpha, st, nullptr, nullptr);
    if ((rc = stage_ok("mlp"))) return rc;
    launch_aev_bwd(ws, n, m.ac, virial ? 1 : 0, st);
    if ((rc = stage_ok("aev_bwd"))) return rc;
    launch_finalize_e(ws, n, mb.e_row, m.md.E, ws.row_cap, m.ebias, st);
  }
  CU_TRY(cudaGetLastError());
  int status[4] = {0, 0, 0, 0};
  CU_TRY(cudaMemcpyAsync(status, ws.status, sizeof(status), cudaMemcpyDeviceToHost, st));
  CU_TRY(cudaStreamSynchronize(st));
  if (status[0] & kStSpecies) return fail(NNP_ERR_SPECIES, "species index out of range");
  if (status[0] & kStNonFinite) return fail(NNP_ERR_NONFINITE, "non-finite coordinate in the ML region");
  if (status[0] & kStCells)
    return fail(NNP_ERR_CAPACITY, "the cell grid needs more than the " +
                                      std::to_string(2 * (long long)n_atoms + 27) +
                                      " cells (2 n + 27) the scratch array holds");
  if (status[0] & kStCapacity)
    return fail(NNP_ERR_CAPACITY, "an atom has more than " + std::to_string(kNoAllocCapR) +
                                      " radial or " + std::to_string(kNoAllocCapA) +
                                      " angular neighbours (fixed lists of the allocation-free entry point)");
  return NNP_OK;
}

extern "C" int nnp_noalloc_max_atoms(const nnp_handle* h, int64_t* max_atoms) {
  g_err.clear();
  if (!h || !max_atoms) return fail(NNP_ERR_ARG, "null argument");
  const Model& m = *h->model;
  if (m.net == kNetBf16) {
    *max_atoms = 0;
    return NNP_OK;
  }
  // the work space grows with the atom count: the largest count whose carve fits
  Ws ws{};
  MlpBufs mb{};
  long long lo = 0, hi = 1 << 24;
  while (lo < hi) {
    const long long mid = (lo + hi + 1) / 2;
    if (noalloc_carve(m, (int)mid, nullptr, &ws, &mb) <= kNoAllocBytes) lo = mid;
    else hi = mid - 1;
  }
  *max_atoms = lo;
  return NNP_OK;
}
