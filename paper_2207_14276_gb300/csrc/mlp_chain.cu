// Fused per-network chain of the per-species networks (paper Eq. 2 and Sec.
// "ANI models") on the 5th-generation tensor cores.
//
// For one 128-row tile of one species segment and one ensemble member e, the
// layers after the first and their backward to the first layer's output run in
// one CTA, the intermediate activations held in shared memory instead of HBM:
//   L2  z2 = h1 W2^T + b2,  h2 = CELU(z2)          A: the h1 tile, by TMA
//   L3  z3 = h2 W3^T + b3,  h3 = CELU(z3)          A: h2 in shared memory
//       E_row += h3 . w4,   delta3 = w4 CELU'(z3)
//   B3  delta2 = (delta3 W3) CELU'(z2)             A: delta3 in shared memory
//   B2  delta1 = (delta2 W2) CELU'(z1)             A: delta2 in shared memory,
//       written over h1 (CELU'(z1) = 1 for h1 > 0, 1 + h1/alpha otherwise)
// The first layer (K = AEV length) and the last backward GEMM (K = E h1, all
// members at once) stay in the layer GEMM kernel (mlp_tc.cu).
//
// Roles (one CTA per SM, persistent over the (member, row tile) list):
//   warp 12       TMA producer: 32-wide K slices (64-byte swizzle) of the h1
//                 tile and of each layer's weights into a ring of stages
//   warp 13       MMA issuer: tcgen05.mma kind::f16 (M = 128, N = layer width)
//                 into one of two 256-column TMEM accumulators
//   warps 0-11    epilogue: warp w reads TMEM lanes 32 (w % 4).. (its rows) and
//                 every third 16-column chunk from chunk w / 4; bias, CELU,
//                 the output dot product, CELU' products; writes the next
//                 layer's A operand into shared memory in the 128-byte-swizzled
//                 K-major layout the MMA reads; CELU'(z2) is rebuilt in B3's
//                 epilogue from L2's accumulator, kept in tensor memory.
// SPLIT: every operand as two BF16 parts (x = hi + lo); each K step issues
// A_hi B_hi + A_lo B_hi + A_hi B_lo, and the shared activations keep both parts.
// Every wait is bounded; a CTA that gives up records a timeout in the status
// word, drains what it issued, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "../../include/nnp.h"
#include "mlp.cuh"
#include "tc_util.cuh"

namespace nnp {

namespace {

using namespace tcu;

constexpr int kCBK = 32;                        // K slice of a ring stage (64-byte swizzle)
constexpr int kCEpiWarps = 12;                  // 14 warps: 4 per SM sub-partition, 128 registers
constexpr int kCGroups = kCEpiWarps / 4;         // column groups of the epilogue
constexpr int kCProdWarp = kCEpiWarps, kCMmaWarp = kCEpiWarps + 1;
constexpr int kCThreads = (kCEpiWarps + 2) * 32;
constexpr int kCMaxStages = 8;
constexpr int kCMaxN = 256;                     // widest layer (one TMEM region)
constexpr int kCActBlk = 128 * 128;             // bytes of one 64-column block of a 128-row A tile
constexpr int kCMaxDynSmem = 232448 - 8192;     // 227 KB per block minus static shared memory

struct ChainArgs {
  int h1, h2, h3, E, S;
  const float* b2; const float* b3; const float* w4;   // [E][S][h]
  float* e_row; int e_row_net;                         // [E][rows]
  __nv_bfloat16* H1; __nv_bfloat16* H1l;               // [rows][E h1]; delta1 written over
  float alpha;
  const int* seg_start;
  int* status;
  int stages, stage_bytes, act_bytes;                  // act_bytes: one plane of the activation
  int energy_only;
};

// shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row atoms 512 B apart
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;               // leading byte offset (unused with this swizzle)
  d |= (uint64_t)(512 >> 4) << 32;      // stride byte offset
  d |= (uint64_t)1 << 46;               // descriptor version
  d |= (uint64_t)4 << 61;               // 64-byte swizzle
  return d;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// 16 values of row r, columns c0 .. c0+15 (c0 a multiple of 16), into a 128-row
// K-major activation tile in the 128-byte-swizzled layout (64-column blocks of
// 16 KB; row r at r * 128 bytes; 16-byte chunk j stored at chunk j ^ (r % 8));
// the split path also writes the low parts into the second plane
template <bool SPLIT>
__device__ __forceinline__ void put_act16(uint8_t* act, int act_bytes, int r, int c0,
                                          const float (&v)[16]) {
  uint8_t* row = act + (c0 >> 6) * kCActBlk + r * 128;
  const int j = (c0 & 63) >> 3;
  uint32_t h[8], l[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    h[i] = pack_bf16x2(v[2 * i], v[2 * i + 1]);
    if (SPLIT) {
      const __nv_bfloat162 hb = *reinterpret_cast<const __nv_bfloat162*>(&h[i]);
      const float2 hf = __bfloat1622float2(hb);
      l[i] = pack_bf16x2(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
    }
  }
  const int o0 = ((j ^ (r & 7)) << 4), o1 = (((j + 1) ^ (r & 7)) << 4);
  *reinterpret_cast<uint4*>(row + o0) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(row + o1) = make_uint4(h[4], h[5], h[6], h[7]);
  if (SPLIT) {
    *reinterpret_cast<uint4*>(row + act_bytes + o0) = make_uint4(l[0], l[1], l[2], l[3]);
    *reinterpret_cast<uint4*>(row + act_bytes + o1) = make_uint4(l[4], l[5], l[6], l[7]);
  }
}

__device__ __forceinline__ void load_f16(const float* p, float (&v)[16]) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 t = __ldg(q + k);
    v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
  }
}

// phase p of a tile: 0 = L2, 1 = L3, 2 = B3, 3 = B2
__device__ __forceinline__ void phase_dims(const ChainArgs& g, int ph, int* K, int* N) {
  switch (ph) {
    case 0: *K = g.h1; *N = g.h2; break;
    case 1: *K = g.h2; *N = g.h3; break;
    case 2: *K = g.h3; *N = g.h2; break;
    default: *K = g.h2; *N = g.h1; break;
  }
}

// TMEM region of a phase's accumulator: L2 and B2 in region b, L3 and B3 in
// region 1 - b, b alternating with the tiles a CTA processes.  L2's
// accumulator (z2 - b2) stays in place until B3's epilogue has rebuilt
// CELU'(z2) from it; the next tile's L2 goes to the region L3 and B3 used, so
// it overlaps the last epilogue of this tile.
__device__ __forceinline__ int region_of(int ph, int tc) {
  const int b = tc & 1;
  return (ph == 0 || ph == 3) ? b : 1 - b;
}

template <bool SPLIT>
__global__ void __launch_bounds__(kCThreads, 1)
k_chain_tc(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mA2,
           const __grid_constant__ CUtensorMap mW2, const __grid_constant__ CUtensorMap mW2l,
           const __grid_constant__ CUtensorMap mW3, const __grid_constant__ CUtensorMap mW3l,
           const __grid_constant__ CUtensorMap mW3T, const __grid_constant__ CUtensorMap mW3Tl,
           const __grid_constant__ CUtensorMap mW2T, const __grid_constant__ CUtensorMap mW2Tl,
           ChainArgs g) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kCMaxStages], empty_bar[kCMaxStages];
  __shared__ __align__(8) uint64_t tfull_bar[2], tempty_bar[2], act_bar, part_bar, bias_bar, done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ float part[kCGroups][128];   // per-row partial output dot products, one per column group
  __shared__ __align__(16) float sbias[2][3 * kCMaxN];   // b2 | b3 | w4 of a tile, two tiles
  __shared__ int abort_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kStages = g.stages;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* act = smem + (size_t)kStages * g.stage_bytes;   // activation tile (hi plane, then lo)
  constexpr int kParts = SPLIT ? 2 : 1;
  constexpr int kABytes = 128 * kCBK * 2;                  // one part of an h1 slice
  volatile int* abort_flag = &abort_sh;
  const int n_ph = g.energy_only ? 2 : 4;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kCMaxStages; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&empty_bar[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull_bar[i], 1);
      mbar_init(&tempty_bar[i], kCEpiWarps);
    }
    mbar_init(&act_bar, kCEpiWarps);
    mbar_init(&part_bar, kCEpiWarps);
    mbar_init(&bias_bar, kCEpiWarps);
    mbar_init(&done_bar, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"((uint32_t)(2 * kCMaxN))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  const int row_tiles = g.seg_start[g.S] / kTileM;
  const int T = row_tiles * g.E;

  if (warp == kCProdWarp) {
    if (lane == 0) {
      // ---- TMA producer: the phases' K slices in the order the MMA warp consumes them
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < T && ok; t += gridDim.x) {
        const Tile tl = tile_of(t, 1, row_tiles, g.E, 0, g.seg_start, g.S);
        const int c2 = tl.e * g.S + tl.s;
        for (int ph = 0; ph < n_ph && ok; ++ph) {
          int K, N;
          phase_dims(g, ph, &K, &N);
          const CUtensorMap* mb = ph == 0 ? &mW2 : ph == 1 ? &mW3 : ph == 2 ? &mW3T : &mW2T;
          const CUtensorMap* mbl = ph == 0 ? &mW2l : ph == 1 ? &mW3l : ph == 2 ? &mW3Tl : &mW2Tl;
          const int nk = (K + kCBK - 1) / kCBK;
          const int b_bytes = N * kCBK * 2;
          const int a_part = ph == 0 ? kABytes : 0;
          for (int kb = 0; kb < nk; ++kb, ++it) {
            const int st = it % kStages;
            const unsigned round = it / kStages;
            if (it >= kStages && !mbar_wait(&empty_bar[st], (round - 1) & 1, abort_flag)) { ok = false; break; }
            uint8_t* base = smem + (size_t)st * g.stage_bytes;
            mbar_expect_tx(&full_bar[st], (unsigned)(kParts * (a_part + b_bytes)));
            if (ph == 0) {
              tma_load_3d(base, &mA, &full_bar[st], kb * kCBK, tl.e, tl.m0);
              if (SPLIT) tma_load_3d(base + kABytes, &mA2, &full_bar[st], kb * kCBK, tl.e, tl.m0);
            }
            uint8_t* bb = base + kParts * a_part;
            tma_load_3d(bb, mb, &full_bar[st], kb * kCBK, 0, c2);
            if (SPLIT) tma_load_3d(bb + b_bytes, mbl, &full_bar[st], kb * kCBK, 0, c2);
          }
        }
      }
      // every issued copy has landed before the CTA may exit
      if (*abort_flag)
        for (int k = it - kStages < 0 ? 0 : it - kStages; k < it; ++k)
          mbar_drain(&full_bar[k % kStages], (k / kStages) & 1);
    }
  } else if (warp == kCMmaWarp) {
    if (lane == 0) {
      // ---- MMA issuer
      int it = 0, a_cnt = 0, tc = 0;
      int use[2] = {0, 0};      // accumulations issued into each TMEM region so far
      bool ok = true;
      const uint32_t act_u = smem_u32(act);
      for (int t = blockIdx.x; t < T && ok; t += gridDim.x, ++tc) {
        for (int ph = 0; ph < n_ph && ok; ++ph) {
          const int reg = region_of(ph, tc);
          // the region's previous accumulation has been released by the epilogue
          if (use[reg] >= 1 && !mbar_wait(&tempty_bar[reg], (use[reg] - 1) & 1, abort_flag)) { ok = false; break; }
          if (ph > 0) {
            if (!mbar_wait(&act_bar, a_cnt & 1, abort_flag)) { ok = false; break; }
            ++a_cnt;
          }
          tc_fence_after();
          int K, N;
          phase_dims(g, ph, &K, &N);
          const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
                                 ((uint32_t)(kTileM >> 4) << 24);
          const uint32_t d = tmem + (uint32_t)(reg * kCMaxN);
          const int nk = (K + kCBK - 1) / kCBK;
          const int b_bytes = N * kCBK * 2;
          for (int kb = 0; kb < nk; ++kb, ++it) {
            const int st = it % kStages;
            if (!mbar_wait(&full_bar[st], (it / kStages) & 1, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint32_t base = smem_u32(smem + (size_t)st * g.stage_bytes);
            const uint32_t sb = base + (ph == 0 ? kParts * kABytes : 0);
#pragma unroll
            for (int j = 0; j < kCBK / 16; ++j) {
              const int kk = kb * (kCBK / 16) + j;
              if (kk * 16 >= K) break;
              uint64_t ad, adl = 0;
              if (ph == 0) {
                ad = sw64_desc(base) + (uint64_t)(j * 2);
                if (SPLIT) adl = sw64_desc(base + kABytes) + (uint64_t)(j * 2);
              } else {
                const uint32_t blk = act_u + (uint32_t)((kk >> 2) * kCActBlk);
                ad = sw128_desc(blk) + (uint64_t)((kk & 3) * 2);
                if (SPLIT) adl = sw128_desc(blk + (uint32_t)g.act_bytes) + (uint64_t)((kk & 3) * 2);
              }
              const uint64_t bd = sw64_desc(sb) + (uint64_t)(j * 2);
              umma_bf16(d, ad, bd, idesc, kk > 0 ? 1u : 0u);
              if (SPLIT) {
                const uint64_t bdl = sw64_desc(sb + (uint32_t)b_bytes) + (uint64_t)(j * 2);
                umma_bf16(d, adl, bd, idesc, 1u);
                umma_bf16(d, ad, bdl, idesc, 1u);
              }
            }
            umma_commit(&empty_bar[st]);
          }
          if (ok) umma_commit(&tfull_bar[reg]);
          ++use[reg];
        }
      }
      umma_commit(&done_bar);   // arrives when every MMA issued above has completed
      mbar_drain(&done_bar, 0);
    }
  } else {
    // ---- epilogue: warp w owns TMEM lanes (rows) 32 q.. and the 16-column chunks
    // 16 cg + 48 ci of each layer, taken two at a time (one TMEM wait per pair)
    const int q = warp & 3, cg = warp >> 2;
    const int r = q * 32 + lane;
    const float alpha = g.alpha, inv_alpha = 1.f / g.alpha;
    int pc = 0, tc = 0;
    int fulls[2] = {0, 0};   // accumulations of each TMEM region waited for so far
    bool ok = true;
    for (int t = blockIdx.x; t < T && ok; t += gridDim.x, ++tc) {
      const Tile tl = tile_of(t, 1, row_tiles, g.E, 0, g.seg_start, g.S);
      const int m = tl.m0 + r;
      const size_t es = (size_t)tl.e * g.S + tl.s;
      // this tile's b2, b3 and w4 into shared memory (double-buffered by tile;
      // the loads overlap the first layer's MMAs)
      float* sb = sbias[tc & 1];
      for (int i = threadIdx.x; i < 3 * kCMaxN; i += kCEpiWarps * 32) {
        const int k = i / kCMaxN, c = i - k * kCMaxN;
        float val = 0.f;
        if (k == 0 && c < g.h2) val = __ldg(g.b2 + es * g.h2 + c);
        else if (k == 1 && c < g.h3) val = __ldg(g.b3 + es * g.h3 + c);
        else if (k == 2 && c < g.h3) val = __ldg(g.w4 + es * g.h3 + c);
        sb[i] = val;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&bias_bar);
      for (int ph = 0; ph < n_ph && ok; ++ph) {
        const int reg = region_of(ph, tc);
        int K, N;
        phase_dims(g, ph, &K, &N);
        const size_t orow = (size_t)m * ((size_t)g.E * g.h1) + (size_t)tl.e * g.h1;
        // B2: the stored h1 of the first chunk pair, fetched before the wait
        uint4 pre[2][2][2];
        if (ph == 3) {
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int c0 = cg * 16 + u * 48;
            if (c0 < N) {
              const uint4* h4 = reinterpret_cast<const uint4*>(g.H1 + orow + c0);
              pre[u][0][0] = h4[0]; pre[u][0][1] = h4[1];
              if (SPLIT) {
                const uint4* l4 = reinterpret_cast<const uint4*>(g.H1l + orow + c0);
                pre[u][1][0] = l4[0]; pre[u][1][1] = l4[1];
              }
            }
          }
        }
        if (!mbar_wait(&tfull_bar[reg], fulls[reg] & 1, abort_flag)) { ok = false; break; }
        ++fulls[reg];
        if (ph == 0 && !mbar_wait(&bias_bar, tc & 1, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(reg * kCMaxN);
        // B3: L2's accumulator z2 - b2, still in the other region
        const uint32_t tz2 = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(region_of(0, tc) * kCMaxN);
        float dot = 0.f;
#pragma unroll
        for (int cp = 0; cp < 3; ++cp) {
          const int c0a = cg * 16 + cp * 96, c0b = c0a + 48;
          if (c0a >= N) break;
          const bool two = c0b < N;
          if (ph == 3 && cp > 0) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int c0 = c0a + u * 48;
              if (c0 < N) {
                const uint4* h4 = reinterpret_cast<const uint4*>(g.H1 + orow + c0);
                pre[u][0][0] = h4[0]; pre[u][0][1] = h4[1];
                if (SPLIT) {
                  const uint4* l4 = reinterpret_cast<const uint4*>(g.H1l + orow + c0);
                  pre[u][1][0] = l4[0]; pre[u][1][1] = l4[1];
                }
              }
            }
          }
          float vv[2][16];
          if (ph == 2) {
            // delta2 = acc * CELU'(z2), z2 = (L2 accumulator) + b2, one chunk at a time
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              if (u == 1 && !two) break;
              const int c0 = c0a + u * 48;
              float z[16];
              tmem_ld16x2(trow + (uint32_t)c0, tz2 + (uint32_t)c0, vv[0], z);
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                const float z2 = z[i] + sb[c0 + i];
                vv[0][i] *= z2 > 0.f ? 1.f : __expf(z2 * inv_alpha);
              }
              put_act16<SPLIT>(act, g.act_bytes, r, c0, vv[0]);   // delta2
            }
            continue;
          }
          if (two) tmem_ld16x2(trow + (uint32_t)c0a, trow + (uint32_t)c0b, vv[0], vv[1]);
          else tmem_ld16(trow + (uint32_t)c0a, vv[0]);
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            if (u == 1 && !two) break;
            const int c0 = c0a + u * 48;
            float (&v)[16] = vv[u];
            if (ph == 0) {
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                const float z = v[i] + sb[c0 + i];
                v[i] = z > 0.f ? z : alpha * (__expf(z * inv_alpha) - 1.f);
              }
              put_act16<SPLIT>(act, g.act_bytes, r, c0, v);
            } else if (ph == 1) {
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                const float z = v[i] + sb[kCMaxN + c0 + i];
                const float w = sb[2 * kCMaxN + c0 + i];
                const float ez = __expf(z * inv_alpha);
                dot = fmaf(z > 0.f ? z : alpha * (ez - 1.f), w, dot);
                v[i] = w * (z > 0.f ? 1.f : ez);   // delta3
              }
              if (!g.energy_only) put_act16<SPLIT>(act, g.act_bytes, r, c0, v);
            } else {
              // CELU'(z1) from the stored h1 (= hi + lo on the split path)
              float a[16];
              {
                const uint32_t wv[8] = {pre[u][0][0].x, pre[u][0][0].y, pre[u][0][0].z, pre[u][0][0].w,
                                        pre[u][0][1].x, pre[u][0][1].y, pre[u][0][1].z, pre[u][0][1].w};
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                  const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&wv[i]));
                  a[2 * i] = f.x; a[2 * i + 1] = f.y;
                }
              }
              if (SPLIT) {
                const uint32_t wv[8] = {pre[u][1][0].x, pre[u][1][0].y, pre[u][1][0].z, pre[u][1][0].w,
                                        pre[u][1][1].x, pre[u][1][1].y, pre[u][1][1].z, pre[u][1][1].w};
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                  const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&wv[i]));
                  a[2 * i] += f.x; a[2 * i + 1] += f.y;
                }
              }
#pragma unroll
              for (int i = 0; i < 16; ++i) v[i] *= (a[i] > 0.f) ? 1.f : fmaf(a[i], inv_alpha, 1.f);
              uint32_t hw[8], lw[8];
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                hw[i] = pack_bf16x2(v[2 * i], v[2 * i + 1]);
                if (SPLIT) {
                  const float2 hf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&hw[i]));
                  lw[i] = pack_bf16x2(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
                }
              }
              uint4* dh = reinterpret_cast<uint4*>(g.H1 + orow + c0);
              dh[0] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
              dh[1] = make_uint4(hw[4], hw[5], hw[6], hw[7]);
              if (SPLIT) {
                uint4* dl = reinterpret_cast<uint4*>(g.H1l + orow + c0);
                dl[0] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                dl[1] = make_uint4(lw[4], lw[5], lw[6], lw[7]);
              }
            }
          }
        }
        // release the accumulations this epilogue was the last to read: L3's after
        // its epilogue, L2's and B3's after B3's epilogue, B2's after its own (an
        // energy-only tile releases L2's and L3's after theirs)
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if (g.energy_only || ph == 1 || ph == 3) mbar_arrive(&tempty_bar[reg]);
          if (ph == 2) {
            mbar_arrive(&tempty_bar[reg]);
            mbar_arrive(&tempty_bar[region_of(0, tc)]);
          }
        }
        const bool writes_act = ph == 0 || ph == 2 || (ph == 1 && !g.energy_only);
        if (writes_act) fence_proxy_async_smem();   // generic writes -> tensor-core reads
        if (ph == 1) {
          // the column groups' partial dot products of each row -> e_row
          part[cg][r] = dot;
          __syncwarp();
          if (lane == 0) mbar_arrive(&part_bar);
          if (cg == 0) {
            if (!mbar_wait(&part_bar, pc & 1, abort_flag)) { ok = false; }
            else g.e_row[(size_t)tl.e * g.e_row_net + m] = part[0][r] + part[1][r] + part[2][r];
          }
          ++pc;
        }
        if (writes_act) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&act_bar);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicOr(g.status, kStTimeout);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)(2 * kCMaxN))
                 : "memory");
}

struct ChainPlan {
  CUtensorMap mA, mA2, mW2, mW2l, mW3, mW3l, mW3T, mW3Tl, mW2T, mW2Tl;
  ChainArgs a;
  dim3 grid;
  size_t smem;
  bool split;
};

}  // namespace

// Set-up of the fused chain for a work arena: tensor maps of h1 and of the
// per-member weights, stage ring size.  Returns null (and the unfused layers
// are used) where the widths do not fit: every width a multiple of 16 and at
// most 256, and the shared-memory ring at least two stages deep.
void* chain_prepare(const MlpDims& md, const MlpWeights& mw, const MlpBufs& mb, int row_cap, bool split) {
  if (!encode_fn() || !mw.W2_h || !mb.H1) return nullptr;
  if (split && (!mw.W2_l || !mb.H1l)) return nullptr;
  const int h1 = md.h1, h2 = md.h2, h3 = md.h3, E = md.E, S = md.S;
  for (int h : {h1, h2, h3})
    if (h % 16 || h > kCMaxN || h < 16) return nullptr;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return nullptr;
  ChainPlan* p = new ChainPlan{};
  p->split = split;
  const int parts = split ? 2 : 1;
  const int act_w = std::max(h2, h3);
  const int act_bytes = ((act_w + 63) / 64) * kCActBlk;
  int stage = 0;
  stage = std::max(stage, 128 * kCBK * 2 + h2 * kCBK * 2);   // L2: h1 slice + W2 slice
  stage = std::max(stage, h3 * kCBK * 2);                    // L3
  stage = std::max(stage, h2 * kCBK * 2);                    // B3
  stage = std::max(stage, h1 * kCBK * 2);                    // B2
  stage *= parts;
  stage = (stage + 1023) / 1024 * 1024;
  const long long room = (long long)kCMaxDynSmem - 1024 - (long long)parts * act_bytes;
  const int stages = (int)std::min<long long>(kCMaxStages, room / stage);
  if (stages < 2) { delete p; return nullptr; }
  const uint64_t R = (uint64_t)row_cap;
  const auto swz = CU_TENSOR_MAP_SWIZZLE_64B;
  // h1 tile: dims (h1, E, rows), box (32, 1, 128)
  bool ok = make_map(&p->mA, mb.H1, h1, E, R, h1, (uint64_t)E * h1, 1, kTileM, kCBK, swz);
  p->mA2 = p->mA;
  if (split) ok = ok && make_map(&p->mA2, mb.H1l, h1, E, R, h1, (uint64_t)E * h1, 1, kTileM, kCBK, swz);
  // weights [E S][N][K]: dims (K, N, E S), box (32, N, 1)
  auto wmap = [&](CUtensorMap* m, const void* base, int K, int N) {
    return make_map(m, base, K, N, (uint64_t)E * S, K, (uint64_t)K * N, (uint32_t)N, 1, kCBK, swz);
  };
  ok = ok && wmap(&p->mW2, mw.W2_h, h1, h2) && wmap(&p->mW3, mw.W3_h, h2, h3) &&
       wmap(&p->mW3T, mw.W3T_h, h3, h2) && wmap(&p->mW2T, mw.W2T_h, h2, h1);
  p->mW2l = p->mW2; p->mW3l = p->mW3; p->mW3Tl = p->mW3T; p->mW2Tl = p->mW2T;
  if (split)
    ok = ok && wmap(&p->mW2l, mw.W2_l, h1, h2) && wmap(&p->mW3l, mw.W3_l, h2, h3) &&
         wmap(&p->mW3Tl, mw.W3T_l, h3, h2) && wmap(&p->mW2Tl, mw.W2T_l, h2, h1);
  if (!ok) { delete p; return nullptr; }
  ChainArgs& a = p->a;
  a.h1 = h1; a.h2 = h2; a.h3 = h3; a.E = E; a.S = S;
  a.b2 = mw.b2; a.b3 = mw.b3; a.w4 = mw.w4;
  a.e_row = mb.e_row; a.e_row_net = row_cap;
  a.H1 = static_cast<__nv_bfloat16*>(mb.H1);
  a.H1l = static_cast<__nv_bfloat16*>(mb.H1l);
  a.stages = stages; a.stage_bytes = stage; a.act_bytes = act_bytes;
  p->smem = (size_t)stages * stage + (size_t)parts * act_bytes + 1024;
  const int row_tiles = (row_cap + kTileM - 1) / kTileM;
  p->grid = dim3((unsigned)std::max(1, std::min(row_tiles * E, sms)));
  const void* fn = split ? (const void*)k_chain_tc<true> : (const void*)k_chain_tc<false>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return nullptr;
  }
  return p;
}

void chain_release(void* plan) { delete static_cast<ChainPlan*>(plan); }

void launch_chain(void* plan, const Ws& ws, float alpha, bool energy_only, cudaStream_t st) {
  ChainPlan* p = static_cast<ChainPlan*>(plan);
  ChainArgs a = p->a;
  a.alpha = alpha;
  a.seg_start = ws.seg_start;
  a.status = ws.status;
  a.energy_only = energy_only ? 1 : 0;
#define NNP_CHAIN_LAUNCH(SPLIT_)                                                               \
  k_chain_tc<SPLIT_><<<p->grid, kCThreads, p->smem, st>>>(p->mA, p->mA2, p->mW2, p->mW2l, p->mW3,   \
                                                         p->mW3l, p->mW3T, p->mW3Tl, p->mW2T,      \
                                                         p->mW2Tl, a)
  if (p->split) NNP_CHAIN_LAUNCH(true);
  else NNP_CHAIN_LAUNCH(false);
#undef NNP_CHAIN_LAUNCH
}

}  // namespace nnp
