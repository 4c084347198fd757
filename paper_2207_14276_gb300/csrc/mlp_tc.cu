// Tensor-core path of the per-species networks (paper Eq. 2): BF16 operands,
// FP32 accumulation in tensor memory, on the 5th-generation tensor cores.
//
// A persistent CTA (one or two per SM) walks a static list of 128-row x n_tile
// output tiles of one layer GEMM
//   C[m, n] = sum_k A[m, e*K + k] * B_{e,s}[n, k]
// for the species s of the tile's 128-row segment and the ensemble member e.
//   warp 8   TMA producer: 64-wide K slices of A and B into a ring of shared
//            memory stages (128-byte swizzle), completion on mbarriers
//   warp 9   MMA issuer: tcgen05.mma kind::f16 (M = 128, N = n_tile, K = 16)
//            into one of two TMEM accumulators; tcgen05.commit frees a stage
//            and, after the tile's last K slice, hands the accumulator over
//   warps 0-7 epilogue: warp w reads accumulator rows 32 (w % 4).. and every
//            other 16-column chunk (w / 4 picks which); bias, CELU, the width-1
//            output layer as a dot product, and in the backward the product
//            with CELU'(z) rebuilt from the stored activation (1 for h > 0,
//            1 + h/alpha otherwise); each 32-row x 16-column chunk goes through
//            a staging slot in shared memory to a TMA store (BF16, or FP32 for
//            dE/dG); then it releases the accumulator to the MMA warp.
// With two accumulators the epilogue of one tile overlaps the MMAs of the next.
// The N tiles of a row tile are adjacent in the tile order (concurrent CTAs
// share the row tile of A in L2).
// Every mbarrier wait is bounded; a CTA that gives up sets the status word,
// drains the copies and MMAs it issued, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "../../include/nnp.h"
#include "mlp.cuh"
#include "tc_util.cuh"

namespace nnp {

// the fused per-network chain (mlp_chain.cu)
void* chain_prepare(const MlpDims& md, const MlpWeights& mw, const MlpBufs& mb, int row_cap, bool split);
void chain_release(void* plan);
void launch_chain(void* plan, const Ws& ws, float alpha, bool energy_only, cudaStream_t st);

namespace {

using namespace tcu;

constexpr int kBM = 128;
constexpr int kBK = 64;           // bf16 elements per K slice (one 128-byte swizzle row)
constexpr int kEpiWarps = 8;
constexpr int kProdWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1;
constexpr int kThreads = (kEpiWarps + 2) * 32;
constexpr int kMaxStages = 4;
// dynamic shared memory limit: the 227 KB per block minus the kernel's static
// shared memory (barriers) and some headroom
constexpr int kMaxDynSmem = 232448 - 2048;
// output staging of an epilogue warp: slots of 32 rows x 16 columns (BF16 high
// part at 0 and low part at 1 KB, or FP32), each written out by one TMA store
constexpr int kSlotBytes = 2048;

struct TcArgs {
  int N, K, n_tile, n_k, tmem_cols, stages, nets;
  int a_c1_per_e;       // A map coordinate 1 = e * a_c1_per_e (net slice)
  int b_c2_per_e;       // B map coordinate 2 = e * b_c2_per_e + s
  uint32_t idesc;
  int epi;
  const float* bias; long long bias_s, bias_e;
  const float* w4; long long w4_s, w4_e;
  void* out; int ldo; int out_net;          // bf16 (or fp32 for kEpiStore)
  void* out2;                               // split path: low parts of out (same layout)
  const void* aux; int ld_aux; int aux_net; // bf16 stored activation (kEpiMul)
  const void* aux2;                         // split path: low parts of aux
  float* e_row; int e_row_net;
  float alpha;
  const int* seg_start;
  int S;
  int* status;
  // sparse AEV rows (null: dense): the live 64-column slices of each 128-row
  // tile; the first layer reads only those K slices, the last backward layer
  // skips the N tiles with none of them
  const uint32_t* kmask;
  const uint32_t* nmask;
  int n_slot;            // output staging slots per epilogue warp (1 or 2)
  int aux_tma;           // kEpiMul, split path: the stored activation's boxes come by TMA
};

// which N tile of a row tile the last backward layer computes (all without nmask)
__device__ __forceinline__ bool ntile_live(const TcArgs& g, int m0, int n0) {
  if (!g.nmask) return true;
  const uint32_t m = g.nmask[m0 >> 7];
  const int a = n0 >> 6, b = (n0 + g.n_tile - 1) >> 6;
  const uint32_t span = (b - a >= 31) ? ~0u : ((2u << (b - a)) - 1u);
  return ((m >> a) & span) != 0u;
}

// One 32-row x 16-column chunk of an epilogue warp's output, through shared
// memory: every lane writes its row's 16 values into the warp's staging slot,
// then lane 0 stores the box with TMA (full-line writes, where direct stores of
// one row per lane would send 32 scattered 32-byte pieces per instruction).
// OUT: 0 BF16, 1 BF16 high and low parts (to / to2), 2 FP32.
template <int OUT>
__device__ __forceinline__ void stage_store(uint8_t* slot, const float (&v)[16], int lane,
                                            const CUtensorMap* to, const CUtensorMap* to2, int x,
                                            int y) {
  if (OUT == 2) {
    float4* d = reinterpret_cast<float4*>(slot + lane * 64);
#pragma unroll
    for (int k = 0; k < 4; ++k) d[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  } else {
    uint32_t wh[8], wl[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
      wh[i] = *reinterpret_cast<const uint32_t*>(&h);
      if (OUT == 1) {
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
        wl[i] = *reinterpret_cast<const uint32_t*>(&l);
      }
    }
    uint4* dh = reinterpret_cast<uint4*>(slot + lane * 32);
    dh[0] = make_uint4(wh[0], wh[1], wh[2], wh[3]);
    dh[1] = make_uint4(wh[4], wh[5], wh[6], wh[7]);
    if (OUT == 1) {
      uint4* dl = reinterpret_cast<uint4*>(slot + 1024 + lane * 32);
      dl[0] = make_uint4(wl[0], wl[1], wl[2], wl[3]);
      dl[1] = make_uint4(wl[4], wl[5], wl[6], wl[7]);
    }
  }
  fence_async_smem();
  __syncwarp();
  if (lane == 0) {
    tma_store_2d(to, slot, x, y);
    if (OUT == 1) tma_store_2d(to2, slot + 1024, x, y);
    bulk_commit();
  }
}

// AUXT (kEpiMul on the split path with TcArgs::aux_tma set): the stored
// activation comes by TMA into shared memory instead of register prefetches
template <int EPI, bool SPLIT, bool AUXT = false>
__global__ void __launch_bounds__(kThreads, 1)
k_gemm_tc(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
          const __grid_constant__ CUtensorMap ta2, const __grid_constant__ CUtensorMap tb2,
          const __grid_constant__ CUtensorMap to, const __grid_constant__ CUtensorMap to2,
          const __grid_constant__ CUtensorMap tx, const __grid_constant__ CUtensorMap tx2,
          TcArgs g) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kMaxStages], empty_bar[kMaxStages];
  __shared__ __align__(8) uint64_t tfull_bar[2], tempty_bar[2], done_bar;
  __shared__ __align__(8) uint64_t aux_bar[kEpiWarps];   // per epilogue warp: its TMA'd aux boxes
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kStages = g.stages;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int a_bytes = kBM * kBK * 2, b_bytes = g.n_tile * kBK * 2;
  constexpr int kParts = SPLIT ? 2 : 1;
  const int stage_bytes = kParts * (a_bytes + b_bytes);   // multiple of 1024
  // after the ring: the epilogue warps' staging slots, then (CELU layers) per
  // epilogue warp the bias and output-layer weights of its columns of a tile
  uint8_t* stg = smem + kStages * stage_bytes;
  float* epi_sh = reinterpret_cast<float*>(stg + kEpiWarps * g.n_slot * kSlotBytes);
  // (kEpiMul with aux_tma) per epilogue warp: its chunks of the stored activation,
  // 2 KB each (high part at 0, low part at 1 KB, 32 rows x 16 columns)
  const int aux_chunks = (g.n_tile / 16 + 1) / 2;
  uint8_t* aux_sm = stg + kEpiWarps * g.n_slot * kSlotBytes;
  volatile int* abort_flag = &abort_sh;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kMaxStages; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&empty_bar[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull_bar[i], 1);
      mbar_init(&tempty_bar[i], kEpiWarps);
    }
    mbar_init(&done_bar, 1);
    for (int i = 0; i < kEpiWarps; ++i) mbar_init(&aux_bar[i], 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"((uint32_t)(2 * g.tmem_cols))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  // tiles: (net, row tile, N tile) with the N tiles innermost; the row tiles
  // counted from the device-side segment table
  const int row_tiles = g.seg_start[g.S] / kBM;
  const int n_tiles_n = (g.N + g.n_tile - 1) / g.n_tile;
  const int T = n_tiles_n * row_tiles * g.nets;

  if (warp == kProdWarp) {
    if (lane == 0) {
      // ---- TMA producer
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < T && ok; t += gridDim.x) {
        const Tile tl = tile_of(t, n_tiles_n, row_tiles, g.nets, g.n_tile, g.seg_start, g.S);
        if (!ntile_live(g, tl.m0, tl.n0)) continue;
        const uint32_t km = g.kmask ? g.kmask[tl.m0 >> 7] : ~0u;
        const int a_c1 = tl.e * g.a_c1_per_e, b_c2 = tl.e * g.b_c2_per_e + tl.s;
        for (int kb = 0; kb < g.n_k; ++kb) {
          if (!((km >> kb) & 1u)) continue;   // an all-zero K slice of the tile
          const int st = it % kStages;
          const unsigned round = it / kStages;
          if (it >= kStages && !mbar_wait(&empty_bar[st], (round - 1) & 1, abort_flag)) { ok = false; break; }
          uint8_t* sa = smem + st * stage_bytes;
          uint8_t* sb = sa + kParts * a_bytes;
          mbar_expect_tx(&full_bar[st], (unsigned)stage_bytes);
          tma_load_3d(sa, &ta, &full_bar[st], kb * kBK, a_c1, tl.m0);
          tma_load_3d(sb, &tb, &full_bar[st], kb * kBK, tl.n0, b_c2);
          if (SPLIT) {
            tma_load_3d(sa + a_bytes, &ta2, &full_bar[st], kb * kBK, a_c1, tl.m0);
            tma_load_3d(sb + b_bytes, &tb2, &full_bar[st], kb * kBK, tl.n0, b_c2);
          }
          ++it;   // copies issued so far
        }
      }
      // every issued copy has landed before the CTA may exit
      if (*abort_flag)
        for (int k = it - kStages < 0 ? 0 : it - kStages; k < it; ++k)
          mbar_drain(&full_bar[k % kStages], (k / kStages) & 1);
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      // ---- MMA issuer
      int it = 0, j = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < T && ok; t += gridDim.x) {
        const Tile tl = tile_of(t, n_tiles_n, row_tiles, g.nets, g.n_tile, g.seg_start, g.S);
        if (!ntile_live(g, tl.m0, tl.n0)) continue;
        const uint32_t km = g.kmask ? g.kmask[tl.m0 >> 7] : ~0u;
        const int ab = j & 1;
        if (j >= 2 && !mbar_wait(&tempty_bar[ab], ((j >> 1) - 1) & 1, abort_flag)) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(ab * g.tmem_cols);
        bool first_k = true;
        for (int kb = 0; kb < g.n_k; ++kb) {
          if (!((km >> kb) & 1u)) continue;
          const int st = it % kStages;
          if (!mbar_wait(&full_bar[st], (it / kStages) & 1, abort_flag)) { ok = false; break; }
          ++it;
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + st * stage_bytes);
          const uint32_t sb = sa + kParts * a_bytes;
          const uint64_t ad = sw128_desc(sa), bd = sw128_desc(sb);
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            umma_bf16(d, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), g.idesc,
                      (!first_k || kk > 0) ? 1u : 0u);
            if (SPLIT) {
              const uint64_t adl = sw128_desc(sa + a_bytes), bdl = sw128_desc(sb + b_bytes);
              umma_bf16(d, adl + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), g.idesc, 1u);
              umma_bf16(d, ad + (uint64_t)(kk * 2), bdl + (uint64_t)(kk * 2), g.idesc, 1u);
            }
          }
          umma_commit(&empty_bar[st]);
          first_k = false;
        }
        if (ok) umma_commit(&tfull_bar[ab]);
        ++j;
      }
      umma_commit(&done_bar);   // arrives when every MMA issued above has completed
      mbar_drain(&done_bar, 0);
    }
  } else {
    // ---- epilogue: warp w owns accumulator rows 32 (w % 4).. and every other
    // 16-column chunk starting at chunk w / 4
    const int q = warp & 3, half = warp >> 2;
    const float alpha = g.alpha, inv_alpha = 1.f / g.alpha;
    constexpr int kOut = EPI == kEpiStore ? 2 : SPLIT ? 1 : 0;
    // BF16 forward layers store straight from registers (measured faster there:
    // 32 bytes per row and chunk; the split and backward layers gain from the
    // staged TMA stores)
    constexpr bool kDirect = !SPLIT && (EPI == kEpiCelu || EPI == kEpiCeluDot);
    uint8_t* my_slots = stg + warp * g.n_slot * kSlotBytes;
    float* my_epi = epi_sh + warp * 2 * 128;
    int n_st = 0;   // chunks this warp has stored
    int j = 0;
    constexpr int kMaxChunks = 256 / 32;   // 16-column chunks of one warp per tile
    for (int t = blockIdx.x; t < T; t += gridDim.x) {
      const Tile tl = tile_of(t, n_tiles_n, row_tiles, g.nets, g.n_tile, g.seg_start, g.S);
      if (!ntile_live(g, tl.m0, tl.n0)) continue;
      const int ab = j & 1;
      const int m = tl.m0 + q * 32 + lane;
      const bool row_ok = NNP_IN_BOUNDS(g.status, kSiteGemmRow, m, g.seg_start[g.S]);
      // the backward's stored activations do not depend on the MMAs: their loads
      // are issued before the wait for the accumulator
      // (the split path also prefetches the low parts)
      // (the first kPD chunks; each later chunk's load is issued when the chunk
      // kPD before it has been used, which bounds the registers they hold)
      constexpr bool kPre = (EPI == kEpiMul);
      constexpr int kPD = SPLIT ? 4 : kMaxChunks;
      uint4 pre[kPre ? kPD : 1][2];
      uint4 prel[kPre && SPLIT ? kPD : 1][2];
      const size_t oa = (size_t)m * g.ld_aux + (size_t)tl.e * g.aux_net + tl.n0;
      const __nv_bfloat16* arow = kPre ? static_cast<const __nv_bfloat16*>(g.aux) + oa : nullptr;
      const __nv_bfloat16* lrow = (kPre && SPLIT) ? static_cast<const __nv_bfloat16*>(g.aux2) + oa : nullptr;
      constexpr bool aux_tma = SPLIT && kPre && AUXT;
      uint8_t* my_aux = aux_sm + warp * aux_chunks * 2048;
      auto fetch_aux = [&](int ci) {
        const int c0 = half * 16 + 32 * ci;
        if (kPre && !aux_tma && row_ok && c0 < g.n_tile && tl.n0 + c0 < g.N) {
          const uint4* src = reinterpret_cast<const uint4*>(arow + c0);
          pre[ci % kPD][0] = src[0];
          pre[ci % kPD][1] = src[1];
          if (SPLIT) {
            const uint4* srl = reinterpret_cast<const uint4*>(lrow + c0);
            prel[ci % kPD][0] = srl[0];
            prel[ci % kPD][1] = srl[1];
          }
        }
      };
      if (kPre) {
#pragma unroll
        for (int ci = 0; ci < kPD; ++ci) fetch_aux(ci);
      }
      if (aux_tma && lane == 0) {
        // this tile's boxes of the stored activation (high and low parts) into
        // the warp's buffer; the warp's reads of the previous tile's boxes are
        // done (it passed the __syncwarp before releasing that accumulator)
        fence_async_smem();
        unsigned bytes = 0;
        for (int ci = 0; ci < aux_chunks; ++ci) {
          const int c0 = half * 16 + 32 * ci;
          if (c0 < g.n_tile && tl.n0 + c0 < g.N) bytes += 2048;
        }
        mbar_expect_tx(&aux_bar[warp], bytes);
        for (int ci = 0; ci < aux_chunks; ++ci) {
          const int c0 = half * 16 + 32 * ci;
          if (c0 < g.n_tile && tl.n0 + c0 < g.N) {
            const int x = tl.e * g.aux_net + tl.n0 + c0, y = tl.m0 + q * 32;
            tma_load_2d(my_aux + ci * 2048, &tx, &aux_bar[warp], x, y);
            tma_load_2d(my_aux + ci * 2048 + 1024, &tx2, &aux_bar[warp], x, y);
          }
        }
      }
      // the bias (and output-layer weights) of this warp's columns, also fetched
      // before the wait: lane l holds entries l + 32 i of the warp's 16-column chunks
      float bpre[4] = {0.f, 0.f, 0.f, 0.f}, wpre[4] = {0.f, 0.f, 0.f, 0.f};
      if (EPI == kEpiCelu || EPI == kEpiCeluDot) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int jj = lane + 32 * i, c0 = half * 16 + 32 * (jj >> 4), n = tl.n0 + c0 + (jj & 15);
          if (c0 < g.n_tile && n < g.N) {
            bpre[i] = __ldg(g.bias + tl.e * g.bias_e + tl.s * g.bias_s + n);
            if (EPI == kEpiCeluDot) wpre[i] = __ldg(g.w4 + tl.e * g.w4_e + tl.s * g.w4_s + n);
          }
        }
      }
      if (!mbar_wait(&tfull_bar[ab], (j >> 1) & 1, abort_flag)) {
        if (aux_tma) mbar_drain(&aux_bar[warp], j & 1);   // the boxes in flight land first
        break;
      }
      if (aux_tma && !mbar_wait(&aux_bar[warp], j & 1, abort_flag)) {
        mbar_drain(&aux_bar[warp], j & 1);
        break;
      }
      if (EPI == kEpiCelu || EPI == kEpiCeluDot) {
        __syncwarp();   // the previous tile's reads of the warp's bias slots are done
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          my_epi[lane + 32 * i] = bpre[i];
          my_epi[128 + lane + 32 * i] = wpre[i];
        }
        __syncwarp();
      }
      tc_fence_after();
      const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * g.tmem_cols);
      float dot = 0.f;
#pragma unroll(kPre ? kMaxChunks : 1)
      for (int ci = 0; ci < kMaxChunks; ++ci) {
        const int c0 = half * 16 + 32 * ci;
        if (c0 >= g.n_tile) break;
        const int n = tl.n0 + c0;
        float v[16];
        tmem_ld16(trow + (uint32_t)c0, v);
        if (n >= g.N) continue;
        if (EPI == kEpiCelu || EPI == kEpiCeluDot) {
          float b[16];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float4 t4 = *reinterpret_cast<const float4*>(&my_epi[ci * 16 + 4 * k]);
            b[4 * k] = t4.x; b[4 * k + 1] = t4.y; b[4 * k + 2] = t4.z; b[4 * k + 3] = t4.w;
          }
          float w4[16];
          if (EPI == kEpiCeluDot) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const float4 t4 = *reinterpret_cast<const float4*>(&my_epi[128 + ci * 16 + 4 * k]);
              w4[4 * k] = t4.x; w4[4 * k + 1] = t4.y; w4[4 * k + 2] = t4.z; w4[4 * k + 3] = t4.w;
            }
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float z = v[i] + b[i];
            const float ez = __expf(z * inv_alpha);
            const float h = z > 0.f ? z : alpha * (ez - 1.f);
            if (EPI == kEpiCeluDot) {
              dot = fmaf(h, w4[i], dot);
              v[i] = w4[i] * (z > 0.f ? 1.f : ez);   // delta3 = w4 * CELU'(z)
            } else {
              v[i] = h;   // CELU' is rebuilt from h where it is needed
            }
          }
        } else if (EPI == kEpiMul) {
          // aux holds the layer's stored activation h = CELU(z): CELU'(z) = 1 for h > 0,
          // 1 + h / alpha otherwise (exp(z/alpha) = 1 + h/alpha on that branch)
          float a[16];
          if (aux_tma) {   // the boxes in shared memory: this lane's row, 32 bytes per part
            const uint4* sh = reinterpret_cast<const uint4*>(my_aux + ci * 2048 + lane * 32);
            const uint4* sl = reinterpret_cast<const uint4*>(my_aux + ci * 2048 + 1024 + lane * 32);
            const uint4 q4[4] = {sh[0], sh[1], sl[0], sl[1]};
            const uint32_t* w = reinterpret_cast<const uint32_t*>(q4);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[i]));
              const float2 fl = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[8 + i]));
              a[2 * i] = f.x + fl.x;
              a[2 * i + 1] = f.y + fl.y;
            }
          } else {
            const uint32_t* w = reinterpret_cast<const uint32_t*>(pre[kPre ? ci % kPD : 0]);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[i]));
              a[2 * i] = f.x;
              a[2 * i + 1] = f.y;
            }
          }
          if (SPLIT && !aux_tma) {
            // the stored activation h = hi + lo (about 16 significant bits)
            const uint32_t* wl = reinterpret_cast<const uint32_t*>(prel[kPre && SPLIT ? ci % kPD : 0]);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&wl[i]));
              a[2 * i] += f.x;
              a[2 * i + 1] += f.y;
            }
          }
          if (ci + kPD < kMaxChunks) fetch_aux(ci + kPD);   // the slot just read is free
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] *= (a[i] > 0.f) ? 1.f : fmaf(a[i], inv_alpha, 1.f);
        }
        if (kDirect && !row_ok) continue;   // bounds-checked build only
        if (!row_ok) {   // bounds-checked build only: a row past the segments stays zero
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = 0.f;
        }
        if (kDirect) {
          store_bf16x16(static_cast<__nv_bfloat16*>(g.out) + (size_t)m * g.ldo +
                            (size_t)tl.e * g.out_net + n, v);
          continue;
        }
        // the chunk through the next staging slot, once the store that last used
        // it has read it
        uint8_t* slot = my_slots + (n_st % g.n_slot) * kSlotBytes;
        if (lane == 0) {
          if (g.n_slot == 2) bulk_wait_read<1>();
          else bulk_wait_read<0>();
        }
        __syncwarp();
        stage_store<kOut>(slot, v, lane, &to, &to2, tl.e * g.out_net + n, tl.m0 + q * 32);
        ++n_st;
      }
      // the two warps of a row each add their half of the output-layer dot product
      // (e_row starts at zero; a sum of two terms does not depend on their order)
      if (EPI == kEpiCeluDot && row_ok) atomicAdd(g.e_row + (size_t)tl.e * g.e_row_net + m, dot);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty_bar[ab]);
      ++j;
    }
    if (lane == 0) bulk_wait_all();   // every output store has completed
  }
  tc_fence_before();
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicOr(g.status, kStTimeout);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)(2 * g.tmem_cols))
                 : "memory");
}

// Failure-path check of the bounded waits: one thread waits (with the limit
// given) on an mbarrier whose phase nothing completes, gives up, and records
// the timeout in the status word exactly as k_gemm_tc does.
__global__ void k_wait_probe(int* status, unsigned limit) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_sh;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  abort_sh = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  bool ok = false;
  for (unsigned it = 0; it < limit && !ok; ++it) ok = mbar_try_wait(&bar, 0);
  if (!ok) atomicOr(status, kStTimeout);
}

// ---------------------------------------------------------------- host side
struct TcGemmPlan {
  CUtensorMap ta, tb, ta2, tb2;   // ta2 / tb2: low parts (split path; copies of ta / tb otherwise)
  CUtensorMap to, to2;            // output (32-row x 16-column boxes); to2: low parts of a split output
  CUtensorMap tx, tx2;            // stored activation of a split kEpiMul layer (same boxes)
  TcArgs a;
  dim3 grid;
  size_t smem;
  int stage_id;
};

struct TcState {
  std::vector<TcGemmPlan> plans;
  void* aev_h = nullptr;
  const float* aev = nullptr;
  float* e_row = nullptr;
  int row_cap = 0, Dp = 0, E = 1;
  bool split = false;
  void* chain = nullptr;     // fused L2 -> L3 -> B3 -> B2 (null: the four layer GEMMs)
  bool use_chain = true;
  ~TcState() {
    if (chain) chain_release(chain);
  }
};

int pick_n_tile(int N, int tiles_per_col, bool single, int sms) {
  // the output-layer dot product needs the whole row in one tile; otherwise the
  // widest multiple of 16 up to 256 that divides N, narrowed while the tiles
  // would not cover every SM
  if (single) return N <= 256 ? N : 256;
  int nt = 16;
  for (int c = 256; c >= 16; c -= 16)
    if (N % c == 0) { nt = c; break; }
  while (tiles_per_col * (N / nt) < sms && nt % 32 == 0 && nt > 64) nt /= 2;
  return nt;
}

int tmem_cols_for(int n_tile) {
  int c = 32;
  while (c < n_tile) c <<= 1;
  return c;
}

}  // namespace

int mlp_tc_prepare(const MlpDims& md, const MlpWeights& mw, const MlpBufs& mb, int row_cap,
                   const float* aev, float* dEdG, bool split, void** state_out) {
  *state_out = nullptr;
  if (!encode_fn()) return NNP_ERR_CUDA;
  if (!mw.W1cat_h || !mb.aev_h) return NNP_ERR_ARG;
  if (split && (!mw.W1cat_l || !mb.aev_l || !mb.H1l || !mb.H2l || !mb.d3l)) return NNP_ERR_ARG;
  TcState* st = new TcState;
  st->split = split;
  st->aev_h = mb.aev_h;
  st->aev = aev;
  st->e_row = mb.e_row;
  st->row_cap = row_cap;
  st->Dp = md.Dp;
  st->E = md.E;
  const int S = md.S, E = md.E, Dp = md.Dp, h1 = md.h1, h2 = md.h2, h3 = md.h3;
  const uint64_t R = (uint64_t)row_cap;
  const int row_tiles = (row_cap + kBM - 1) / kBM;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    delete st;
    return NNP_ERR_CUDA;
  }
  struct L {
    int stage, epi, N, K, nets;
    const void* A; uint64_t a_d0, a_d1, a_st1, a_st2;
    const void* B; uint64_t b_d0, b_d1, b_d2;
    int b_c2_per_e;
    const float* bias; long long bias_s, bias_e;
    const float* w4; long long w4_s, w4_e;
    void* out; int ldo, out_net; void* out2; const void* aux; int ld_aux, aux_net;
    // split path: low parts of A, B, out and aux
    const void* A2; const void* B2; void* out_lo; const void* aux_lo;
  };
  std::vector<L> layers = {
      // L1: AEV x [W1 of all members]^T
      {3, kEpiCelu, E * h1, Dp, 1, mb.aev_h, (uint64_t)Dp, 1, (uint64_t)Dp, (uint64_t)Dp,
       mw.W1cat_h, (uint64_t)Dp, (uint64_t)E * h1, (uint64_t)S, 0, mw.b1cat, (long long)E * h1, 0,
       nullptr, 0, 0, mb.H1, E * h1, 0, mb.D1, nullptr, 0, 0,
       mb.aev_l, mw.W1cat_l, mb.H1l, nullptr},
      // L2 per member
      {4, kEpiCelu, h2, h1, E, mb.H1, (uint64_t)h1, (uint64_t)E, (uint64_t)h1, (uint64_t)E * h1,
       mw.W2_h, (uint64_t)h1, (uint64_t)h2, (uint64_t)E * S, S, mw.b2, h2, (long long)S * h2,
       nullptr, 0, 0, mb.H2, E * h2, h2, mb.D2, nullptr, 0, 0,
       mb.H1l, mw.W2_l, mb.H2l, nullptr},
      // L3 + output dot
      {5, kEpiCeluDot, h3, h2, E, mb.H2, (uint64_t)h2, (uint64_t)E, (uint64_t)h2, (uint64_t)E * h2,
       mw.W3_h, (uint64_t)h2, (uint64_t)h3, (uint64_t)E * S, S, mw.b3, h3, (long long)S * h3,
       mw.w4, h3, (long long)S * h3, mb.d3, E * h3, h3, nullptr, nullptr, 0, 0,
       mb.H2l, mw.W3_l, mb.d3l, nullptr},
      // B3: delta2 = (delta3 W3) * CELU'(z2) from H2, written over H2
      {6, kEpiMul, h2, h3, E, mb.d3, (uint64_t)h3, (uint64_t)E, (uint64_t)h3, (uint64_t)E * h3,
       mw.W3T_h, (uint64_t)h3, (uint64_t)h2, (uint64_t)E * S, S, nullptr, 0, 0, nullptr, 0, 0,
       mb.H2, E * h2, h2, nullptr, mb.H2, E * h2, h2,
       mb.d3l, mw.W3T_l, mb.H2l, mb.H2l},
      // B2: delta1 = (delta2 W2) * CELU'(z1) from H1, written over H1
      {7, kEpiMul, h1, h2, E, mb.H2, (uint64_t)h2, (uint64_t)E, (uint64_t)h2, (uint64_t)E * h2,
       mw.W2T_h, (uint64_t)h2, (uint64_t)h1, (uint64_t)E * S, S, nullptr, 0, 0, nullptr, 0, 0,
       mb.H1, E * h1, h1, nullptr, mb.H1, E * h1, h1,
       mb.H2l, mw.W2T_l, mb.H1l, mb.H1l},
      // B1: dE/dG = [delta1_e] [W1_e / E]   (K = E*h1), FP32 output
      {8, kEpiStore, Dp, E * h1, 1, mb.H1, (uint64_t)E * h1, 1, (uint64_t)E * h1, (uint64_t)E * h1,
       mw.W1Tcat_h, (uint64_t)E * h1, (uint64_t)Dp, (uint64_t)S, 0, nullptr, 0, 0, nullptr, 0, 0,
       dEdG, Dp, 0, nullptr, nullptr, 0, 0,
       mb.H1l, mw.W1Tcat_l, nullptr, nullptr},
  };
  for (const L& l : layers) {
    TcGemmPlan p{};
    const bool single = (l.epi == kEpiCeluDot);
    int nt = pick_n_tile(l.N, row_tiles * l.nets, single, sms);
    // wide split backward layers that multiply by CELU' (N >= 256): half-width N
    // tiles, so that the ring, the output slots and the TMA'd boxes of the stored
    // activation fit in shared memory together (measured: B2 of the 8-network
    // model 0.524 -> 0.401 ms; at N = 192 the narrower tiles cost more than the
    // loads gain, 0.326 -> 0.335 ms, and B3 keeps its register prefetch)
    const bool aux_tma = split && l.epi == kEpiMul && l.N % 32 == 0 && l.N >= 256 && l.N / 2 <= 256;
    if (aux_tma) nt = l.N / 2;
    // the last backward layer skips N tiles without a live AEV slice (sparse
    // rows): on the split path 128-wide tiles follow the rows' live columns twice
    // as closely as 256-wide ones (a water row's live columns are the first 128;
    // measured on the 8-network model: 0.442 -> 0.365 ms; the BF16 path, whose
    // MMAs are a third as long, keeps 256: 0.187 against 0.210 ms)
    if (split && l.epi == kEpiStore && l.N % 128 == 0 && nt > 128) nt = 128;
    if (nt % 16 != 0 || nt > 256 || (single && nt < l.N)) { delete st; return NNP_ERR_UNSUPPORTED; }
    if (!make_map(&p.ta, l.A, l.a_d0, l.a_d1, R, l.a_st1, l.a_st2, 1, kBM) ||
        !make_map(&p.tb, l.B, l.b_d0, l.b_d1, l.b_d2, l.b_d0, l.b_d0 * l.b_d1, (uint32_t)nt, 1)) {
      delete st;
      return NNP_ERR_CUDA;
    }
    if (split) {
      if (!make_map(&p.ta2, l.A2, l.a_d0, l.a_d1, R, l.a_st1, l.a_st2, 1, kBM) ||
          !make_map(&p.tb2, l.B2, l.b_d0, l.b_d1, l.b_d2, l.b_d0, l.b_d0 * l.b_d1, (uint32_t)nt, 1)) {
        delete st;
        return NNP_ERR_CUDA;
      }
    } else {
      p.ta2 = p.ta;
      p.tb2 = p.tb;
    }
    if (aux_tma) {
      if (!make_map_2d(&p.tx, l.aux, false, (uint64_t)l.ld_aux, R, (uint64_t)l.ld_aux, 16, 32) ||
          !make_map_2d(&p.tx2, l.aux_lo, false, (uint64_t)l.ld_aux, R, (uint64_t)l.ld_aux, 16, 32)) {
        delete st;
        return NNP_ERR_CUDA;
      }
    }
    // the output: [row_cap][ldo] (FP32 dE/dG for the last layer, BF16 otherwise)
    const bool out_fp32 = (l.epi == kEpiStore);
    if (!make_map_2d(&p.to, l.out, out_fp32, (uint64_t)l.ldo, R, (uint64_t)l.ldo, 16, 32) ||
        !make_map_2d(&p.to2, (split && !out_fp32) ? l.out_lo : l.out, out_fp32, (uint64_t)l.ldo, R,
                     (uint64_t)l.ldo, 16, 32)) {
      delete st;
      return NNP_ERR_CUDA;
    }
    if (!aux_tma) {   // unused by the kernel, but passed: any valid map
      p.tx = p.to;
      p.tx2 = p.to2;
    }
    TcArgs& a = p.a;
    a.N = l.N; a.K = l.K; a.n_tile = nt; a.n_k = (l.K + kBK - 1) / kBK;
    a.tmem_cols = tmem_cols_for(nt);
    a.nets = l.nets;
    a.a_c1_per_e = (l.nets > 1) ? 1 : 0;
    a.b_c2_per_e = l.b_c2_per_e;
    a.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(nt >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
    a.epi = l.epi;
    a.bias = l.bias; a.bias_s = l.bias_s; a.bias_e = l.bias_e;
    a.w4 = l.w4; a.w4_s = l.w4_s; a.w4_e = l.w4_e;
    a.out = l.out; a.ldo = l.ldo; a.out_net = l.out_net;
    a.out2 = split ? l.out_lo : nullptr;
    a.aux = l.aux; a.ld_aux = l.ld_aux; a.aux_net = l.aux_net;
    a.aux2 = split ? l.aux_lo : nullptr;
    a.e_row = mb.e_row; a.e_row_net = row_cap;
    // CTAs per SM: as many as the 512 tensor-memory columns hold (two accumulators
    // each), at most two; the shared memory is split between them and never so
    // small that more CTAs could share an SM than its tensor memory holds
    // (the split path holds both parts of A and B per stage; it takes one CTA per
    // SM where two would leave each CTA fewer than two stages)
    const size_t stage_bytes = (size_t)(split ? 2 : 1) * (kBM * kBK * 2 + nt * kBK * 2);
    // besides the ring: the epilogue warps' staging slots and, for the CELU
    // layers, their bias and output-layer weight slots
    const size_t epi_bytes = (l.epi == kEpiCelu || l.epi == kEpiCeluDot) ? kEpiWarps * 2 * 128 * 4
                             : aux_tma ? (size_t)kEpiWarps * ((nt / 16 + 1) / 2) * 2048 : 0;
    auto extra = [&](int slots) { return (size_t)kEpiWarps * slots * kSlotBytes + epi_bytes; };
    auto stages_for = [&](int c, int slots) {
      const size_t budget = std::min((size_t)kMaxDynSmem, (size_t)232448 / c - 2048);
      if (budget < 1024 + extra(slots) + stage_bytes) return 0;
      const int n = (int)std::min<size_t>(kMaxStages, (budget - 1024 - extra(slots)) / stage_bytes);
      return std::min(n, std::max(a.n_k, 1));
    };
    // (the BF16 forward layers store from registers and need no slots)
    const bool direct = !split && (l.epi == kEpiCelu || l.epi == kEpiCeluDot);
    int ctas = std::min(2, 512 / (2 * a.tmem_cols));
    if (split && ctas == 2 && stages_for(2, 1) < std::min(2, a.n_k)) ctas = 1;
    // two staging slots per warp (a chunk's store overlaps the next chunk) unless
    // that would cost a ring stage
    const int slots = direct ? 0 : stages_for(ctas, 2) >= stages_for(ctas, 1) ? 2 : 1;
    const int stages = stages_for(ctas, slots);
    if (stages < 1) { delete st; return NNP_ERR_UNSUPPORTED; }
    a.stages = stages;
    a.n_slot = slots;
    a.aux_tma = aux_tma ? 1 : 0;
    size_t sm = (size_t)stages * stage_bytes + 1024 + extra(slots);
    const size_t floor_sm = 232448 / (size_t)(ctas + 1) + 1;
    p.smem = sm > floor_sm ? sm : floor_sm;
    if (p.smem > (size_t)kMaxDynSmem) { delete st; return NNP_ERR_UNSUPPORTED; }
    const long long tiles = (long long)((l.N + nt - 1) / nt) * row_tiles * l.nets;
    p.grid = dim3((unsigned)std::max(1LL, std::min(tiles, (long long)sms * ctas)));
    p.stage_id = l.stage;
    st->plans.push_back(p);
  }
  const void* fns[9] = {(const void*)k_gemm_tc<kEpiCelu, false>, (const void*)k_gemm_tc<kEpiCeluDot, false>,
                        (const void*)k_gemm_tc<kEpiMul, false>, (const void*)k_gemm_tc<kEpiStore, false>,
                        (const void*)k_gemm_tc<kEpiCelu, true>, (const void*)k_gemm_tc<kEpiCeluDot, true>,
                        (const void*)k_gemm_tc<kEpiMul, true>, (const void*)k_gemm_tc<kEpiStore, true>,
                        (const void*)k_gemm_tc<kEpiMul, true, true>};
  for (const void* fn : fns)
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem) != cudaSuccess) {
      delete st;
      return NNP_ERR_CUDA;
    }
  st->chain = chain_prepare(md, mw, mb, row_cap, split);
  *state_out = st;
  return NNP_OK;
}

void mlp_tc_release(void* state) { delete static_cast<TcState*>(state); }

// whether the layers after the first run as the fused chain (where it is set up)
void mlp_tc_use_chain(void* state, bool on) {
  if (state) static_cast<TcState*>(state)->use_chain = on;
}

void launch_wait_probe(int* status, unsigned limit, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(status, limit);
}

int launch_mlp_tc(const Ws& ws, const MlpDims& md, const MlpWeights& mw, const MlpBufs& mb, float alpha,
                  cudaStream_t st, int* n_launch, StageHook* hook, void* state, bool energy_only,
                  bool skip_l1) {
  (void)mw; (void)mb;
  TcState* s = static_cast<TcState*>(state);
  if (!s) return NNP_ERR_ARG;
  // plans 0-2 are the forward layers, 3-5 the backward to the input; with the
  // fused chain: plan 0 (L1), the chain (L2, L3, B3, B2), plan 5 (B1)
  const bool chain = s->chain && s->use_chain;
  const size_t n_plans = energy_only ? 3 : s->plans.size();
  // sparse AEV rows of this call (the AEV kernel wrote the tile masks)
  const uint32_t* tmask = (ws.row_mask && !skip_l1) ? ws.tile_mask : nullptr;
  for (size_t i = 0; i < n_plans; ++i) {
    if (i == 0 && skip_l1) continue;   // the first layer ran with the AEV kernel
    if (chain && i >= 1 && i <= 4) {
      if (i == 1) {
        if (hook) hook->begin(13);
        launch_chain(s->chain, ws, alpha, energy_only, st);
        if (hook) hook->end();
      }
      continue;
    }
    auto& p = s->plans[i];
    TcArgs a = p.a;
    a.alpha = alpha;
    a.seg_start = ws.seg_start;
    a.S = md.S;
    a.status = ws.status;
    a.kmask = (i == 0) ? tmask : nullptr;                       // L1: live K slices
    a.nmask = (i == s->plans.size() - 1) ? tmask : nullptr;     // B1: live N tiles
    if (hook) hook->begin(p.stage_id);
    // the two epilogue warps of a row add their halves of the output dot product
    if (a.epi == kEpiCeluDot) cudaMemsetAsync(a.e_row, 0, sizeof(float) * (size_t)md.E * a.e_row_net, st);
    // a masked layer skips N tiles by their index within a row tile; with a grid
    // that is a multiple of the N tiles per row tile every CTA would keep one
    // index (and the CTAs of the skipped ones would idle): take a grid coprime
    // with that count
    dim3 grid = p.grid;
    if (a.nmask) {
      const int ntn = (a.N + a.n_tile - 1) / a.n_tile;
      auto gcd = [](int x, int y) { while (y) { const int t = x % y; x = y; y = t; } return x; };
      while (grid.x > 1 && ntn > 1 && gcd((int)grid.x, ntn) != 1) --grid.x;
    }
#define NNP_TC_LAUNCH(EPI_, SPLIT_) \
  k_gemm_tc<EPI_, SPLIT_><<<grid, kThreads, p.smem, st>>>(p.ta, p.tb, p.ta2, p.tb2, p.to, p.to2, p.tx, p.tx2, a)
    if (s->split) {
      switch (a.epi) {
        case kEpiCelu: NNP_TC_LAUNCH(kEpiCelu, true); break;
        case kEpiCeluDot: NNP_TC_LAUNCH(kEpiCeluDot, true); break;
        case kEpiMul:
          if (a.aux_tma)
            k_gemm_tc<kEpiMul, true, true><<<grid, kThreads, p.smem, st>>>(p.ta, p.tb, p.ta2, p.tb2, p.to,
                                                                            p.to2, p.tx, p.tx2, a);
          else
            NNP_TC_LAUNCH(kEpiMul, true);
          break;
        default: NNP_TC_LAUNCH(kEpiStore, true); break;
      }
    } else {
      switch (a.epi) {
        case kEpiCelu: NNP_TC_LAUNCH(kEpiCelu, false); break;
        case kEpiCeluDot: NNP_TC_LAUNCH(kEpiCeluDot, false); break;
        case kEpiMul: NNP_TC_LAUNCH(kEpiMul, false); break;
        default: NNP_TC_LAUNCH(kEpiStore, false); break;
      }
    }
#undef NNP_TC_LAUNCH
    if (hook) hook->end();
  }
  if (n_launch) *n_launch += (chain ? (energy_only ? 2 : 3) : (int)n_plans) - (skip_l1 ? 1 : 0);
  return NNP_OK;
}

}  // namespace nnp
