// Per-species network chain (paper Eq. 2 and Sec. "ANI models"): the layer
// GEMMs over 128-row species segments of the AEV matrix, their fused
// epilogues, and the buffers they use.
#pragma once

#include "nnp_internal.cuh"

namespace nnp {

enum Epi : int {
  kEpiCelu = 0,     // out = CELU(acc + b), out2 = CELU'(acc + b)
  kEpiCeluDot = 1,  // e_row += CELU(acc + b) . w4 ; out = w4 * CELU'(acc + b)
  kEpiMul = 2,      // out = acc * aux
  kEpiStore = 3,    // out = acc
  kEpiStoreMul = 4, // out = acc, out2 = acc * aux
};

// One grouped GEMM: for every 128-row tile of species s and net e = blockIdx.z,
//   C[m, n] = sum_k A[m, e*a_net + k] * B_{e,s}[n, k]      (B row-major [N, K])
struct GemmArgs {
  const void* A; int lda; int a_net;
  const void* B; long long b_s, b_e; int ldb;
  const float* bias; long long bias_s, bias_e;
  const float* w4; long long w4_s, w4_e;
  int N, K;
  void* out; int ldo; int out_net;
  void* out2;            // CELU' output (same layout as out)
  const void* aux; int ld_aux; int aux_net;
  float* e_row; int e_row_net;   // per-net row energies
  int epi;
  float alpha;           // CELU alpha
  const int* seg_start;  // [S+1]
  int S;
};

struct MlpDims {
  int S, E, Dp, h1, h2, h3;
};

// device weights (FP32 layouts; BF16 copies for the tensor-core path)
struct MlpWeights {
  float* W1cat;  float* b1cat;   // [S][E*h1][Dp], [S][E*h1]
  float* W2;     float* b2;      // [E][S][h2][h1], [E][S][h2]
  float* W3;     float* b3;      // [E][S][h3][h2], [E][S][h3]
  float* w4;                     // [E][S][h3]
  float* W3T;                    // [E][S][h2][h3]
  float* W2T;                    // [E][S][h1][h2]
  float* W1Tcat;                 // [S][Dp][E*h1]   (scaled by 1/E)
  float* ebias;                  // [S] mean_e b4 + species shift
  // bf16 copies (same layouts), null for the FP32 path
  void* W1cat_h; void* W2_h; void* W3_h; void* W3T_h; void* W2T_h; void* W1Tcat_h;
  // split path: the low parts w - bf16(w), rounded to bf16 (same layouts)
  void* W1cat_l; void* W2_l; void* W3_l; void* W3T_l; void* W2T_l; void* W1Tcat_l;
};

// activation buffers
struct MlpBufs {
  void* H1;   // [rows][E*h1]  (reused for delta1)
  void* D1;   // [rows][E*h1]
  void* H2;   // [rows][E*h2]  (reused for delta2)
  void* D2;   // [rows][E*h2]
  void* d3;   // [rows][E*h3]
  float* e_row;  // [E][rows]
  void* aev_h;   // bf16 copy of the AEV (tensor-core path)
  // split path: low bf16 parts of the AEV, H1, H2 and d3 (same layouts as the
  // high parts, which are aev_h, H1, H2 and d3)
  void* aev_l; void* H1l; void* H2l; void* d3l;
};

// optional per-stage timing callback of the runtime (events on the stream)
struct StageHook {
  void* h = nullptr;
  void* st = nullptr;
  void* cur = nullptr;
  int cur_id = 0;
  void begin(int id);
  void end();
};

void launch_gemm_fp32(const GemmArgs& g, int row_cap, cudaStream_t st);
void launch_gemm_fp32(const GemmArgs& g, int row_cap, cudaStream_t st, int n_nets);
// the whole FP32 chain of one-network models as a single kernel per 32-row tile
bool mlp_fused_supported(const MlpDims& md);
cudaError_t mlp_fused_ensure_smem(const MlpDims& md);
void launch_mlp_fused(const Ws& ws, const MlpDims& md, const MlpWeights& mw, const MlpBufs& mb,
                      float alpha, bool energy_only, cudaStream_t st);
void launch_mlp_fp32(const Ws& ws, const MlpDims& md, const MlpWeights& mw, const MlpBufs& mb,
                     float alpha, cudaStream_t st, int* n_launch, StageHook* hook,
                     bool energy_only = false);

}  // namespace nnp
