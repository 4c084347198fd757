// FP32 path of the per-species networks (paper Eq. 2) as one kernel: the three
// hidden layers, the width-1 output layer and the backward to the input
// (dE/dG for the force kernel) for a 32-row tile of one species, with every
// activation kept in shared memory.
//
// Per tile (rows m, species s, one network):
//   L1  H1 = CELU(G W1^T + b1)           G streamed from the AEV rows
//   L2  H2 = CELU(H1 W2^T + b2)
//   L3  H3 = CELU(H2 W3^T + b3), e = H3 . w4, D3 = w4 * CELU'(Z3)
//   B3  delta2 = (D3 W3) * CELU'(Z2)      written over H2
//   B2  delta1 = (delta2 W2) * CELU'(Z1)  written over H1
//   B1  dE/dG = delta1 W1                 written to global memory
// CELU'(Z) is rebuilt from the stored activation: 1 for H > 0, else 1 + H/alpha
// (CELU(z) = alpha (exp(z/alpha) - 1) on the negative branch).
//
// Each phase is a 32 x N block product on 8 warps: warp w owns rows 4w..4w+3 of
// the tile and all N columns, a thread an accumulator tile of 4 rows x N/32
// columns.  A lane owns 4 consecutive columns per 128-wide group (then 2 of a
// 64-wide and 1 of a 32-wide remainder), so that a K-slice row of the weights is
// read with 16-byte loads, and the activation operand is a broadcast 16-byte load
// of 4 consecutive k of one row.  Weight K-slices (k-major, from the transposed
// or plain layout as the phase needs) stream through a cp.async ring in shared
// memory, two slices ahead of the one in use: a tile's phases are a chain of ~45
// slices, and one L2 round trip per slice would otherwise set the kernel's
// duration.
#include "mlp.cuh"

namespace nnp {

namespace {

constexpr int kRows = 32;       // rows per CTA
constexpr int kThreads = 256;   // 8 warps, 4 rows of the tile each
constexpr int KS = 32;          // K-slice of one pipeline stage
constexpr int NS = 3;           // stages of the cp.async ring (NS - 1 slices in flight)
constexpr int kOutChunk = 128;  // B1 output columns per pass

struct FusedArgs {
  const float* G;       // AEV rows [row][Dp]
  float* dEdG;          // [row][Dp]
  float* e_row;         // [row] per-row network energy
  const int* seg_start; // [S+1]
  const int* species_count;
  int S, Dp;
  // weights of species 0; species s adds s times the per-species stride
  const float* W1T; long long sW1T;  // [Dp][h1]
  const float* W1;  long long sW1;   // [h1][Dp]
  const float* b1;  long long sb1;
  const float* W2T; long long sW2;   // [h1][h2]
  const float* W2;                   // [h2][h1]
  const float* b2;  long long sb2;
  const float* W3T; long long sW3;   // [h2][h3]
  const float* W3;                   // [h3][h2]
  const float* b3;  long long sb3;
  const float* w4;  long long sw4;
  float alpha;
  int energy_only;
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? 16 : 0;  // 0 source bytes: the 16 bytes are zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
// wait until at most N of this thread's most recent cp.async groups are pending
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ float comp(const float4& v, int q) {
  return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}

__device__ __forceinline__ float celu_f(float z, float alpha, float inv_alpha) {
  return z > 0.f ? z : alpha * (__expf(z * inv_alpha) - 1.f);
}
// CELU' from the activation h = CELU(z)
__device__ __forceinline__ float celu_d_of_h(float h, float inv_alpha) {
  return h > 0.f ? 1.f : fmaf(h, inv_alpha, 1.f);
}

// The columns a lane owns in an N-wide block (N a multiple of 32), in
// accumulator order: 128 g + 4 lane + i (g < Q, i < 4), then 128 Q + 2 lane + i
// (i < 2) if the remainder holds 64 columns, then 128 Q + 64 P + lane.
template <int N>
struct Cols {
  static_assert(N % 32 == 0, "block width");
  static constexpr int C = N / 32;
  static constexpr int Q = N / 128;
  static constexpr int P = (N % 128) >= 64 ? 1 : 0;
  static constexpr int S1 = (N % 64) ? 1 : 0;
  // v[c] = row[col(c)] for c < C   (row 16-byte aligned; v may be longer)
  template <int CM>
  __device__ static __forceinline__ void load(float (&v)[CM], const float* row, int lane) {
#pragma unroll
    for (int g = 0; g < Q; ++g) {
      const float4 t = *reinterpret_cast<const float4*>(row + 128 * g + 4 * lane);
      v[4 * g] = t.x; v[4 * g + 1] = t.y; v[4 * g + 2] = t.z; v[4 * g + 3] = t.w;
    }
    if (P) {
      const float2 t = *reinterpret_cast<const float2*>(row + 128 * Q + 2 * lane);
      v[4 * Q] = t.x; v[4 * Q + 1] = t.y;
    }
    if (S1) v[C - 1] = row[128 * Q + 64 * P + lane];
  }
  template <int CM>
  __device__ static __forceinline__ void store(const float (&v)[CM], float* row, int lane) {
#pragma unroll
    for (int g = 0; g < Q; ++g)
      *reinterpret_cast<float4*>(row + 128 * g + 4 * lane) =
          make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
    if (P) *reinterpret_cast<float2*>(row + 128 * Q + 2 * lane) = make_float2(v[4 * Q], v[4 * Q + 1]);
    if (S1) row[128 * Q + 64 * P + lane] = v[C - 1];
  }
};

constexpr int RPW = 4;   // rows per warp: warp w owns rows 4w..4w+3 of the tile

// acc[r][c] = sum_k A[row 4w + r][k] * B[k][n0 + col(c)] over k < K (K a multiple
// of KS).  A: shared [32][lda] (AG = false) or global rows Ag[row][ldg] starting
// at the tile (AG = true, staged through As).  B: global [K][ldb]; columns
// n0 + j >= Nv read as zero.
template <int N, bool AG>
__device__ __forceinline__ void block_gemm(float (&acc)[RPW][N / 32], const float* A, int lda,
                                           const float* Ag, int ldg, float* As, int K,
                                           const float* B, int ldb, int n0, int Nv, float* Bs) {
  constexpr int C = N / 32;
  constexpr int kVec = KS * N / 4;  // float4s per B slice
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
#pragma unroll
  for (int r = 0; r < RPW; ++r)
#pragma unroll
    for (int c = 0; c < C; ++c) acc[r][c] = 0.f;
  auto issue = [&](int k0, int buf) {
    float* bs = Bs + buf * KS * N;
#pragma unroll
    for (int i = 0; i < (kVec + kThreads - 1) / kThreads; ++i) {
      const int idx = tid + i * kThreads;
      if (kVec % kThreads == 0 || idx < kVec) {
        const int row = idx / (N / 4), col = (idx % (N / 4)) * 4;
        const bool ok = n0 + col < Nv;
        cp_async16(bs + row * N + col, B + (size_t)(k0 + row) * ldb + (ok ? n0 + col : 0), ok);
      }
    }
    if (AG && tid < kRows * KS / 4) {  // 32 rows x KS k of the AEV: one float4 per thread
      const int row = tid / (KS / 4), q = tid % (KS / 4);
      cp_async16(As + buf * kRows * (KS + 4) + row * (KS + 4) + q * 4,
                 Ag + (size_t)row * ldg + k0 + q * 4, true);
    }
    cp_async_commit();
  };
  // NS-stage ring: slice sl lives in buffer sl % NS; NS - 1 slices are issued
  // ahead, and every iteration commits one group (empty past the end) so that
  // "at most NS - 2 groups pending" always means "slice sl has landed"
  const int n_slices = K / KS;
#pragma unroll
  for (int i = 0; i < NS - 1; ++i) {
    if (i < n_slices) issue(i * KS, i);
    else cp_async_commit();
  }
  for (int sl = 0; sl < n_slices; ++sl) {
    const int buf = sl % NS;
    cp_async_wait<NS - 2>();
    __syncthreads();   // slice sl visible to all; every warp is done with slice sl - 1
    if (sl + NS - 1 < n_slices) issue((sl + NS - 1) * KS, (sl + NS - 1) % NS);
    else cp_async_commit();
    const float* bs = Bs + buf * KS * N;
    const float* arow = AG ? As + buf * kRows * (KS + 4) + (w * RPW) * (KS + 4)
                           : A + (size_t)(w * RPW) * lda + sl * KS;
    const int lds = AG ? KS + 4 : lda;
#pragma unroll
    for (int kk = 0; kk < KS; kk += 4) {
      float4 a[RPW];
#pragma unroll
      for (int r = 0; r < RPW; ++r) a[r] = *reinterpret_cast<const float4*>(arow + r * lds + kk);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float b[C];
        Cols<N>::load(b, bs + (kk + q) * N, lane);
#pragma unroll
        for (int r = 0; r < RPW; ++r) {
          const float av = comp(a[r], q);
#pragma unroll
          for (int c = 0; c < C; ++c) acc[r][c] = fmaf(av, b[c], acc[r][c]);
        }
      }
    }
  }
  cp_async_wait<0>();   // only empty groups remain; none may straddle the next phase
  __syncthreads();  // every warp is done with Bs/As (and with A) before they are reused
}

constexpr int cmax(int a, int b) { return a > b ? a : b; }

template <int N1, int N2, int N3>
struct Smem {
  static constexpr int ld1 = N1 + 4, ld2 = N2 + 4, ld3 = N3 + 4;
  static constexpr int H1 = 0, H2 = H1 + kRows * ld1, H3 = H2 + kRows * ld2;
  static constexpr int As = H2;  // the AEV stage of L1 lives where H2/H3 go later
  static constexpr int Bs = H3 + kRows * ld3;
  static constexpr int floats = Bs + NS * KS * cmax(cmax(N1, N2), cmax(N3, kOutChunk));
  static_assert(NS * kRows * (KS + 4) <= kRows * (ld2 + ld3), "A stage overlay");
};

// L1/L2 epilogue: H[row][col] = CELU(acc + b[col])
template <int N>
__device__ __forceinline__ void store_celu(float (&acc)[RPW][N / 32], const float* bias, float* H,
                                           int ld, int w, int lane, float alpha, float inv_alpha) {
  constexpr int C = N / 32;
  float b[C];
  Cols<N>::load(b, bias, lane);
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
#pragma unroll
    for (int c = 0; c < C; ++c) acc[r][c] = celu_f(acc[r][c] + b[c], alpha, inv_alpha);
    Cols<N>::store(acc[r], H + (w * RPW + r) * ld, lane);
  }
}

// B3/B2 epilogue: H[row][col] = acc * CELU'(z) rebuilt from the stored H
template <int N>
__device__ __forceinline__ void store_delta(float (&acc)[RPW][N / 32], float* H, int ld, int w,
                                            int lane, float inv_alpha) {
  constexpr int C = N / 32;
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    float* row = H + (w * RPW + r) * ld;
    float hv[C];
    Cols<N>::load(hv, row, lane);
#pragma unroll
    for (int c = 0; c < C; ++c) acc[r][c] *= celu_d_of_h(hv[c], inv_alpha);
    Cols<N>::store(acc[r], row, lane);
  }
}

template <int N1, int N2, int N3, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_mlp_fused(FusedArgs a) {
  using L = Smem<N1, N2, N3>;
  extern __shared__ __align__(16) float smf[];
  const int m0 = blockIdx.x * kRows;
  const int total = a.seg_start[a.S];
  if (m0 >= total) return;
  int s = 0;
  while (s + 1 < a.S && m0 >= a.seg_start[s + 1]) ++s;
  if (m0 - a.seg_start[s] >= a.species_count[s]) return;  // padding rows only
  const int Dp = a.Dp;
  float* H1 = smf + L::H1;  // [32][ld1]
  float* H2 = smf + L::H2;  // [32][ld2]
  float* H3 = smf + L::H3;  // [32][ld3]
  float* As = smf + L::As;  // [NS][32][KS+4], during L1 only
  float* Bs = smf + L::Bs;  // [NS][KS][N]
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float alpha = a.alpha, inv_alpha = 1.f / a.alpha;

  // ---- L1
  {
    float acc[RPW][N1 / 32];
    block_gemm<N1, true>(acc, nullptr, 0, a.G + (size_t)m0 * Dp, Dp, As, Dp,
                         a.W1T + s * a.sW1T, N1, 0, N1, Bs);
    store_celu<N1>(acc, a.b1 + s * a.sb1, H1, L::ld1, w, lane, alpha, inv_alpha);
  }
  __syncthreads();
  // ---- L2
  {
    float acc[RPW][N2 / 32];
    block_gemm<N2, false>(acc, H1, L::ld1, nullptr, 0, nullptr, N1, a.W2T + s * a.sW2, N2, 0, N2, Bs);
    store_celu<N2>(acc, a.b2 + s * a.sb2, H2, L::ld2, w, lane, alpha, inv_alpha);
  }
  __syncthreads();
  // ---- L3 and the output layer: e = H3 . w4, D3 = w4 * CELU'(Z3)
  {
    constexpr int C = N3 / 32;
    float acc[RPW][C];
    block_gemm<N3, false>(acc, H2, L::ld2, nullptr, 0, nullptr, N2, a.W3T + s * a.sW3, N3, 0, N3, Bs);
    float b[C], w4[C], dot[RPW];
    Cols<N3>::load(b, a.b3 + s * a.sb3, lane);
    Cols<N3>::load(w4, a.w4 + s * a.sw4, lane);
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      dot[r] = 0.f;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const float z = acc[r][c] + b[c];
        dot[r] = fmaf(celu_f(z, alpha, inv_alpha), w4[c], dot[r]);
        acc[r][c] = w4[c] * (z > 0.f ? 1.f : __expf(z * inv_alpha));
      }
      Cols<N3>::store(acc[r], H3 + (w * RPW + r) * L::ld3, lane);
    }
#pragma unroll
    for (int r = 0; r < RPW; ++r)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dot[r] += __shfl_xor_sync(0xffffffffu, dot[r], o);
    if (lane < RPW) {
      float v = dot[0];
#pragma unroll
      for (int r = 1; r < RPW; ++r) v = lane == r ? dot[r] : v;
      a.e_row[m0 + w * RPW + lane] = v;
    }
  }
  if (a.energy_only) return;
  __syncthreads();
  // ---- B3: delta2 = (D3 W3) * CELU'(Z2), over H2
  {
    float acc[RPW][N2 / 32];
    block_gemm<N2, false>(acc, H3, L::ld3, nullptr, 0, nullptr, N3, a.W3 + s * a.sW3, N2, 0, N2, Bs);
    store_delta<N2>(acc, H2, L::ld2, w, lane, inv_alpha);
  }
  __syncthreads();
  // ---- B2: delta1 = (delta2 W2) * CELU'(Z1), over H1
  {
    float acc[RPW][N1 / 32];
    block_gemm<N1, false>(acc, H2, L::ld2, nullptr, 0, nullptr, N2, a.W2 + s * a.sW2, N1, 0, N1, Bs);
    store_delta<N1>(acc, H1, L::ld1, w, lane, inv_alpha);
  }
  __syncthreads();
  // ---- B1: dE/dG = delta1 W1, 128 columns per pass (Dp a multiple of 128)
  const float* W1 = a.W1 + s * a.sW1;
  for (int n0 = 0; n0 < Dp; n0 += kOutChunk) {
    float acc[RPW][kOutChunk / 32];
    block_gemm<kOutChunk, false>(acc, H1, L::ld1, nullptr, 0, nullptr, N1, W1, Dp, n0, Dp, Bs);
#pragma unroll
    for (int r = 0; r < RPW; ++r)
      Cols<kOutChunk>::store(acc[r], a.dEdG + (size_t)(m0 + w * RPW + r) * Dp + n0, lane);
  }
}

struct Variant {
  int h1, h2, h3;
  void (*fn)(FusedArgs);
  size_t smem;
};
const Variant kVariants[] = {
    // 160-128-96 (4-species model), two CTAs per SM
    {160, 128, 96, k_mlp_fused<160, 128, 96, 2>, Smem<160, 128, 96>::floats * sizeof(float)},
    // 256-192-160 (7-species model)
    {256, 192, 160, k_mlp_fused<256, 192, 160, 1>, Smem<256, 192, 160>::floats * sizeof(float)},
};

const Variant* find_variant(const MlpDims& md) {
  if (md.E != 1 || md.Dp % kOutChunk) return nullptr;
  for (const Variant& v : kVariants)
    if (v.h1 == md.h1 && v.h2 == md.h2 && v.h3 == md.h3) return &v;
  return nullptr;
}

}  // namespace

bool mlp_fused_supported(const MlpDims& md) {
  const Variant* v = find_variant(md);
  return v != nullptr;
}

cudaError_t mlp_fused_ensure_smem(const MlpDims& md) {
  const Variant* v = find_variant(md);
  if (!v) return cudaSuccess;
  const int need = (int)v->smem;
  cudaFuncAttributes attr;
  cudaError_t e = cudaFuncGetAttributes(&attr, (const void*)v->fn);
  if (e != cudaSuccess) return e;
  if (attr.maxDynamicSharedSizeBytes < need)
    e = cudaFuncSetAttribute((const void*)v->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
  return e;
}

void launch_mlp_fused(const Ws& ws, const MlpDims& md, const MlpWeights& mw, const MlpBufs& mb,
                      float alpha, bool energy_only, cudaStream_t st) {
  const Variant* v = find_variant(md);
  FusedArgs a{};
  a.G = ws.aev;
  a.dEdG = ws.dEdG;
  a.e_row = mb.e_row;
  a.seg_start = ws.seg_start;
  a.species_count = ws.species_count;
  a.S = md.S; a.Dp = md.Dp;
  // with one network the concatenated layouts are per-species blocks
  a.W1T = mw.W1Tcat; a.sW1T = (long long)md.Dp * md.h1;
  a.W1 = mw.W1cat;   a.sW1 = (long long)md.h1 * md.Dp;
  a.b1 = mw.b1cat;   a.sb1 = md.h1;
  a.W2T = mw.W2T;    a.sW2 = (long long)md.h2 * md.h1;
  a.W2 = mw.W2;
  a.b2 = mw.b2;      a.sb2 = md.h2;
  a.W3T = mw.W3T;    a.sW3 = (long long)md.h3 * md.h2;
  a.W3 = mw.W3;
  a.b3 = mw.b3;      a.sb3 = md.h3;
  a.w4 = mw.w4;      a.sw4 = md.h3;
  a.alpha = alpha;
  a.energy_only = energy_only ? 1 : 0;
  const int grid = (ws.row_cap + kRows - 1) / kRows;
  void* args[] = {&a};
  cudaLaunchKernel((const void*)v->fn, dim3(grid), dim3(kThreads), args, v->smem, st);
}

}  // namespace nnp
