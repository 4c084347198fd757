// FP32 path of the per-species networks (paper Eq. 2): a tiled SIMT GEMM with
// fused epilogues, run over 128-row species segments of the AEV matrix (a
// 64-row tile never straddles two species).
//
// Forward per layer: Z = H W^T + b, H' = CELU(Z), D = CELU'(Z) (kept for the
// backward).  The last hidden layer's epilogue also forms the atomic energy
// e = H3 . w4 (the width-1 output layer as a dot product) and delta3 = w4 * D3.
// Backward to the input (dE/dG for the force kernel): delta_{l-1} =
// (delta_l W_l) * D_{l-1}, and dE/dG = delta1 W1 with the ensemble members
// concatenated along K (weights pre-transposed and pre-scaled by 1/E at create).
#include "mlp.cuh"

namespace nnp {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;
constexpr int TM = 8, TN = 4;                  // outputs per thread
constexpr int kThreads = (BM / TM) * (BN / TN);  // 128

__device__ __forceinline__ float celu_f(float z, float alpha, float inv_alpha) {
  return z > 0.f ? z : alpha * (__expf(z * inv_alpha) - 1.f);
}
__device__ __forceinline__ float celu_d(float z, float inv_alpha) {
  return z > 0.f ? 1.f : __expf(z * inv_alpha);
}

// 64 x 64 output tile per CTA, 128 threads with an 8 x 4 register tile each
// (rows ty*8.., columns tx*4..).  16-wide K slices of A and B are staged
// through registers into a double-buffered, transposed shared-memory copy, so
// each thread reads its 8 rows and 4 columns of one K step as three 16-byte loads.
template <int EPI>
__global__ void __launch_bounds__(kThreads) k_gemm_fp32(GemmArgs g) {
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];
  const int m0 = blockIdx.x * BM;
  const int total = g.seg_start[g.S];
  if (m0 >= total) return;
  int s = 0;
  while (s + 1 < g.S && m0 >= g.seg_start[s + 1]) ++s;
  const int e = blockIdx.z;
  const int n0 = blockIdx.y * BN;
  if (n0 >= g.N) return;
  const float* A = static_cast<const float*>(g.A) + (size_t)e * g.a_net;
  const float* B = static_cast<const float*>(g.B) + e * g.b_e + s * g.b_s;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // loaders: A and B slices are 64 rows x 16 k = 256 float4 each, 2 per thread
  float4 ra[2], rb[2];
  auto load = [&](int k0) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int idx = tid + i * kThreads, r = idx >> 2, q = idx & 3;
      ra[i] = *reinterpret_cast<const float4*>(A + (size_t)(m0 + r) * g.lda + k0 + q * 4);
      rb[i] = (n0 + r < g.N) ? *reinterpret_cast<const float4*>(B + (size_t)(n0 + r) * g.ldb + k0 + q * 4)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int idx = tid + i * kThreads, r = idx >> 2, q = idx & 3;
      As[buf][q * 4 + 0][r] = ra[i].x; As[buf][q * 4 + 1][r] = ra[i].y;
      As[buf][q * 4 + 2][r] = ra[i].z; As[buf][q * 4 + 3][r] = ra[i].w;
      Bs[buf][q * 4 + 0][r] = rb[i].x; Bs[buf][q * 4 + 1][r] = rb[i].y;
      Bs[buf][q * 4 + 2][r] = rb[i].z; Bs[buf][q * 4 + 3][r] = rb[i].w;
    }
  };
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  load(0);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < g.K; k0 += BK) {
    const bool more = k0 + BK < g.K;
    if (more) load(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * TM]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * TM + 4]);
      const float4 bv = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * TN]);
      const float a[TM] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[TN] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
  // ---- epilogue (N is a multiple of 16: a thread's 4 columns are all in or all out)
  const int nb = n0 + tx * TN;
  const bool n_ok = nb < g.N;
  const float alpha = g.alpha, inv_alpha = 1.f / g.alpha;
  if (EPI == kEpiCelu || EPI == kEpiCeluDot) {
    float bias[TN] = {0.f, 0.f, 0.f, 0.f}, w4[TN] = {0.f, 0.f, 0.f, 0.f};
    if (n_ok) {
      const float* bp = g.bias + e * g.bias_e + s * g.bias_s + nb;
      for (int j = 0; j < TN; ++j) bias[j] = bp[j];
      if (EPI == kEpiCeluDot) {
        const float* wp = g.w4 + e * g.w4_e + s * g.w4_s + nb;
        for (int j = 0; j < TN; ++j) w4[j] = wp[j];
      }
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int m = m0 + ty * TM + i;
      float h[TN], dd[TN], dot = 0.f;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const float zz = acc[i][j] + bias[j];
        h[j] = celu_f(zz, alpha, inv_alpha);
        dd[j] = celu_d(zz, inv_alpha);
        dot = fmaf(h[j], w4[j], dot);
      }
      float* o = static_cast<float*>(g.out) + (size_t)m * g.ldo + (size_t)e * g.out_net + nb;
      if (EPI == kEpiCelu) {
        if (n_ok) {
          *reinterpret_cast<float4*>(o) = make_float4(h[0], h[1], h[2], h[3]);
          float* o2 = static_cast<float*>(g.out2) + (size_t)m * g.ldo + (size_t)e * g.out_net + nb;
          *reinterpret_cast<float4*>(o2) = make_float4(dd[0], dd[1], dd[2], dd[3]);
        }
      } else {
        if (n_ok)
          *reinterpret_cast<float4*>(o) =
              make_float4(w4[0] * dd[0], w4[1] * dd[1], w4[2] * dd[2], w4[3] * dd[3]);
        // the 16 threads of a row group hold the row's columns
#pragma unroll
        for (int o2 = 1; o2 < 16; o2 <<= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o2);
        if (tx == 0) atomicAdd(g.e_row + (size_t)e * g.e_row_net + m, dot);
      }
    }
  } else {
    if (!n_ok) return;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int m = m0 + ty * TM + i;
      float v[TN] = {acc[i][0], acc[i][1], acc[i][2], acc[i][3]};
      float* o = static_cast<float*>(g.out) + (size_t)m * g.ldo + (size_t)e * g.out_net + nb;
      if (EPI == kEpiMul || EPI == kEpiStoreMul) {
        const float4 a = *reinterpret_cast<const float4*>(
            static_cast<const float*>(g.aux) + (size_t)m * g.ld_aux + (size_t)e * g.aux_net + nb);
        if (EPI == kEpiStoreMul) {
          *reinterpret_cast<float4*>(o) = make_float4(v[0], v[1], v[2], v[3]);
          o = static_cast<float*>(g.out2) + (size_t)m * g.ldo + (size_t)e * g.out_net + nb;
        }
        v[0] *= a.x; v[1] *= a.y; v[2] *= a.z; v[3] *= a.w;
      }
      *reinterpret_cast<float4*>(o) = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
}

}  // namespace

void launch_gemm_fp32(const GemmArgs& g, int row_cap, cudaStream_t st, int n_nets) {
  dim3 grid((row_cap + BM - 1) / BM, (g.N + BN - 1) / BN, n_nets);
  switch (g.epi) {
    case kEpiCelu: k_gemm_fp32<kEpiCelu><<<grid, kThreads, 0, st>>>(g); break;
    case kEpiCeluDot: k_gemm_fp32<kEpiCeluDot><<<grid, kThreads, 0, st>>>(g); break;
    case kEpiMul: k_gemm_fp32<kEpiMul><<<grid, kThreads, 0, st>>>(g); break;
    case kEpiStoreMul: k_gemm_fp32<kEpiStoreMul><<<grid, kThreads, 0, st>>>(g); break;
    default: k_gemm_fp32<kEpiStore><<<grid, kThreads, 0, st>>>(g); break;
  }
}

void launch_gemm_fp32(const GemmArgs& g, int row_cap, cudaStream_t st) {
  launch_gemm_fp32(g, row_cap, st, 1);
}

// the six GEMMs of one forward + backward-to-input pass over every species
// (one fused kernel where the network shape has a compiled variant)
void launch_mlp_fp32(const Ws& ws, const MlpDims& md, const MlpWeights& mw, const MlpBufs& mb,
                     float alpha, cudaStream_t st, int* n_launch, StageHook* hook,
                     bool energy_only) {
  if (mlp_fused_supported(md)) {  // one kernel for the whole chain
    if (hook) hook->begin(12);
    launch_mlp_fused(ws, md, mw, mb, alpha, energy_only, st);
    if (hook) hook->end();
    if (n_launch) *n_launch += 1;
    return;
  }
  const int E = md.E, S = md.S, Dp = md.Dp, h1 = md.h1, h2 = md.h2, h3 = md.h3;
  const int R = ws.row_cap;
  GemmArgs g{};
  g.alpha = alpha;
  g.seg_start = ws.seg_start;
  g.S = S;
  g.e_row = mb.e_row;
  g.e_row_net = R;
  cudaMemsetAsync(mb.e_row, 0, sizeof(float) * (size_t)E * R, st);
  // L1: all ensemble members at once along N
  g.A = ws.aev; g.lda = Dp; g.a_net = 0;
  g.B = mw.W1cat; g.b_s = (long long)E * h1 * Dp; g.b_e = 0; g.ldb = Dp;
  g.bias = mw.b1cat; g.bias_s = (long long)E * h1; g.bias_e = 0;
  g.N = E * h1; g.K = Dp;
  g.out = mb.H1; g.out2 = mb.D1; g.ldo = E * h1; g.out_net = 0;
  g.epi = kEpiCelu;
  if (hook) hook->begin(3);
  launch_gemm_fp32(g, R, st, 1);
  if (hook) hook->end();
  // L2: per member
  g.A = mb.H1; g.lda = E * h1; g.a_net = h1;
  g.B = mw.W2; g.b_s = (long long)h2 * h1; g.b_e = (long long)S * h2 * h1; g.ldb = h1;
  g.bias = mw.b2; g.bias_s = h2; g.bias_e = (long long)S * h2;
  g.N = h2; g.K = h1;
  g.out = mb.H2; g.out2 = mb.D2; g.ldo = E * h2; g.out_net = h2;
  g.epi = kEpiCelu;
  if (hook) hook->begin(4);
  launch_gemm_fp32(g, R, st, E);
  if (hook) hook->end();
  // L3 + output layer as a dot product; delta3 = w4 * CELU'(Z3)
  g.A = mb.H2; g.lda = E * h2; g.a_net = h2;
  g.B = mw.W3; g.b_s = (long long)h3 * h2; g.b_e = (long long)S * h3 * h2; g.ldb = h2;
  g.bias = mw.b3; g.bias_s = h3; g.bias_e = (long long)S * h3;
  g.w4 = mw.w4; g.w4_s = h3; g.w4_e = (long long)S * h3;
  g.N = h3; g.K = h2;
  g.out = mb.d3; g.out2 = nullptr; g.ldo = E * h3; g.out_net = h3;
  g.epi = kEpiCeluDot;
  if (hook) hook->begin(5);
  launch_gemm_fp32(g, R, st, E);
  if (hook) hook->end();
  if (energy_only) {   // no forces wanted: the backward to the input is skipped
    if (n_launch) *n_launch += 4;
    return;
  }
  // B3: delta2 = (delta3 W3) * D2   (written over H2)
  g.A = mb.d3; g.lda = E * h3; g.a_net = h3;
  g.B = mw.W3T; g.b_s = (long long)h2 * h3; g.b_e = (long long)S * h2 * h3; g.ldb = h3;
  g.N = h2; g.K = h3;
  g.aux = mb.D2; g.ld_aux = E * h2; g.aux_net = h2;
  g.out = mb.H2; g.ldo = E * h2; g.out_net = h2;
  g.epi = kEpiMul;
  if (hook) hook->begin(6);
  launch_gemm_fp32(g, R, st, E);
  if (hook) hook->end();
  // B2: delta1 = (delta2 W2) * D1   (written over H1)
  g.A = mb.H2; g.lda = E * h2; g.a_net = h2;
  g.B = mw.W2T; g.b_s = (long long)h1 * h2; g.b_e = (long long)S * h1 * h2; g.ldb = h2;
  g.N = h1; g.K = h2;
  g.aux = mb.D1; g.ld_aux = E * h1; g.aux_net = h1;
  g.out = mb.H1; g.ldo = E * h1; g.out_net = h1;
  g.epi = kEpiMul;
  if (hook) hook->begin(7);
  launch_gemm_fp32(g, R, st, E);
  if (hook) hook->end();
  // B1: dE/dG = [delta1_e]_e [W1_e / E]_e   (K = E*h1)
  g.A = mb.H1; g.lda = E * h1; g.a_net = 0;
  g.B = mw.W1Tcat; g.b_s = (long long)Dp * E * h1; g.b_e = 0; g.ldb = E * h1;
  g.N = Dp; g.K = E * h1;
  g.out = ws.dEdG; g.ldo = Dp; g.out_net = 0;
  g.epi = kEpiStore;
  if (hook) hook->begin(8);
  launch_gemm_fp32(g, R, st, 1);
  if (hook) hook->end();
  if (n_launch) *n_launch += 7;
}

}  // namespace nnp
