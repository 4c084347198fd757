// Atomic environment vectors (paper Eqs. 3-5) and their backward to forces.
//
// One warp per centre atom.  The geometry of every neighbour of the centre is
// computed once (lane-parallel) and staged in shared memory: (R, f_c) for the
// radial list, (unit vector, R) and (f_c, f_c') for the angular sub-list.
//
// Forward
//   radial  (Eq. 4): two half-warps take alternate neighbours of one species, a
//           lane owns one Gaussian shell r; an xor-16 shuffle adds the halves
//           and lanes 0..15 write the block's 16 features.
//   angular (Eq. 5): lane-per-triplet.  The (j, k) pairs of one unordered
//           species pair are numbered and decoded in closed form; every lane
//           forms the 4 Gaussians of the averaged distance and the 8 angular
//           factors of its pair (two sections per packed FP32x2 instruction)
//           and accumulates all 32 products in registers.
//           A transpose-reduce across the warp (31 shuffles) leaves lane l with
//           feature l = 8a + z of the block: one coalesced 128-byte store.
//   The angular factor uses cos(theta - theta_z) = cos theta cos theta_z +
//   sin theta sin theta_z with sin theta from the cross product (no acos), and
//   (1 + cos(theta - theta_z))^zeta by repeated squaring (integer zeta,
//   specialised at compile time for zeta = 32).
//
// Backward (F = -dE/dr)
//   radial edges: lane-per-neighbour, 16 shells each (two per packed FP32x2
//   instruction).
//   angular: lane-per-pair (j, k) of the centre's angular neighbours, the pairs
//   taken in round-robin order (one round pairs every neighbour at most once).
//   The dE/dG of the species-pair blocks that have pairs is staged in shared
//   memory (feature order, up to 16 blocks).  Each lane contracts its block's
//   32 values to dE/dcos, dE/dRbar and dE/d(f_j f_k), forms dE/du_j and dE/du_k
//   and adds them to per-neighbour accumulators in shared memory: round r into
//   copy r mod (number of copies), so no two lanes of a pass add into the same
//   address.  Afterwards each neighbour receives one vector atomic and the
//   centre one warp-reduced atomic.  Centres with too many angular neighbours
//   or blocks go to a CTA-per-centre kernel.
#include <cuda_bf16.h>

#include <algorithm>

#include "nnp_internal.cuh"
#include "tc_util.cuh"

namespace nnp {

namespace {

constexpr int kWarps = 8;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kPi = 3.14159265358979f;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float fast_exp2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// hardware approximations (relative error of a few 1e-8): square root of the
// squared distance and the sine, reciprocals of distances and of sin(theta)
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// x^e for an integer exponent; compile-time E > 0 unrolls, E == 0 reads e
template <int E>
__device__ __forceinline__ float ipow(float x, int e) {
  if constexpr (E > 0) {
    float r = 1.f, b = x;
#pragma unroll
    for (int k = E; k; k >>= 1) {
      if (k & 1) r *= b;
      if (k > 1) b *= b;
    }
    return r;
  } else {
    float r = 1.f;
    while (e) {
      if (e & 1) r *= x;
      x *= x;
      e >>= 1;
    }
    return r;
  }
}

struct Geo {
  float dx, dy, dz, r;
};

__device__ __forceinline__ Geo pair_geo(const float4& xi, const float4& xj, const SysDev& d) {
  float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
  if (d.in.periodic) {
    float n;
    n = rintf(dx * d.in.inv_box[0]); dx = fmaf(-n, d.in.box_hi[0], dx); dx = fmaf(-n, d.in.box_lo[0], dx);
    n = rintf(dy * d.in.inv_box[1]); dy = fmaf(-n, d.in.box_hi[1], dy); dy = fmaf(-n, d.in.box_lo[1], dy);
    n = rintf(dz * d.in.inv_box[2]); dz = fmaf(-n, d.in.box_hi[2], dz); dz = fmaf(-n, d.in.box_lo[2], dz);
  }
  Geo g;
  g.dx = dx; g.dy = dy; g.dz = dz;
  g.r = sqrt_approx(dx * dx + dy * dy + dz * dz);
  return g;
}

// One lane per entry of a neighbour list: visit(slot, j, geometry) stages entry j.
// A lane takes two entries per pass and issues both gathers before either is used.
template <class Visit>
__device__ __forceinline__ void stage_list(int n, const int* lst, const float4& xi, const SysDev& d,
                                           const Ws& ws, unsigned lane, Visit visit) {
  const float4* xyzq = ws.xyzq;
  for (int t0 = 0; t0 < n; t0 += 64) {
    const int ta = t0 + (int)lane, tb = ta + 32;
    int ja = ta < n ? lst[ta] : -1;
    int jb = tb < n ? lst[tb] : -1;
    if (ja >= 0 && !NNP_IN_BOUNDS(ws.status, kSiteAevNeighbour, ja, ws.totals[0])) ja = -1;
    if (jb >= 0 && !NNP_IN_BOUNDS(ws.status, kSiteAevNeighbour, jb, ws.totals[0])) jb = -1;
    const float4 xa = ja >= 0 ? xyzq[ja] : xi;
    const float4 xb = jb >= 0 ? xyzq[jb] : xi;
    if (ja >= 0) visit(ta, ja, pair_geo(xi, xa, d));
    if (jb >= 0) visit(tb, jb, pair_geo(xi, xb, d));
  }
}

// cosine cutoff (Eq. 3) and its derivative (inv_rc = 1 / rc)
__device__ __forceinline__ float fcut(float r, float rc, float inv_rc) {
  return r < rc ? 0.5f * cospif(r * inv_rc) + 0.5f : 0.f;
}
__device__ __forceinline__ void fcut_both(float r, float rc, float inv_rc, float* f, float* df) {
  if (r < rc) {
    float sn, cs;
    sincospif(r * inv_rc, &sn, &cs);
    *f = 0.5f * cs + 0.5f;
    *df = -0.5f * kPi * inv_rc * sn;
  } else {
    *f = 0.f;
    *df = 0.f;
  }
}

// sin(theta) with theta = acos(k cos_hat): sqrt(1 - k^2 cos_hat^2) written as
// sqrt(|u_j x u_k|^2 + (1 - k^2) cos_hat^2), which keeps full relative accuracy
// for nearly collinear triplets (where 1 - cos^2 cancels)
__device__ __forceinline__ float sin_theta(const float4& a, const float4& b, float chat, float k) {
  const float cx = a.y * b.z - a.z * b.y;
  const float cy = a.z * b.x - a.x * b.z;
  const float cz = a.x * b.y - a.y * b.x;
  const float s2 = cx * cx + cy * cy + cz * cz;
  return sqrt_approx(fmaf(1.f - k * k, chat * chat, s2));
}

// The angular factors of two sections at once (the pair (z, z + 1) of one
// float2): base = 1 + c cos(theta_z) + s sin(theta_z), B = base^zeta, and
// B1 = base^(zeta - 1) where asked for.  Packed FP32x2 multiplies and FMAs (one
// instruction for both sections; each lane is an IEEE FP32 operation).
template <int ZETA>
__device__ __forceinline__ float2 section_pair(const AevConst& ac, int m, float2 c2, float2 s2,
                                               float2* B1 = nullptr) {
  const float2 cz = reinterpret_cast<const float2*>(ac.cos_z)[m];
  const float2 sz = reinterpret_cast<const float2*>(ac.sin_z)[m];
  const float2 base = __ffma2_rn(s2, sz, __ffma2_rn(c2, cz, make_float2(1.f, 1.f)));
  if constexpr (ZETA == 32) {
    float2 p = __fmul2_rn(base, base);   // ^2
    p = __fmul2_rn(p, p);                // ^4
    p = __fmul2_rn(p, p);                // ^8
    p = __fmul2_rn(p, p);                // ^16
    const float2 B = __fmul2_rn(p, p);
    // base >= 1 + cos(15 pi / 16) > 0: base^31 = base^32 / base
    if (B1) *B1 = __fmul2_rn(B, make_float2(rcp_approx(base.x), rcp_approx(base.y)));
    return B;
  } else {
    const float2 b1 = make_float2(ipow<0>(base.x, ac.zeta - 1), ipow<0>(base.y, ac.zeta - 1));
    if (B1) *B1 = b1;
    return __fmul2_rn(b1, base);
  }
}

// per-warp header: species offsets/counts of the radial and angular lists
struct ListHdr {
  int off_r[kMaxSpecies + 1], off_a[kMaxSpecies + 1];
  unsigned live[2];   // backward kernel: angular blocks with triplets (bit q = block q)
};

// dE/dG blocks of a centre held in shared memory by the warp-per-centre backward
// kernel (the blocks with triplets, in block order; a centre with more goes to
// the CTA-per-centre kernel)
constexpr int kGallBlocks = 16;

// float4s of shared memory per warp of the backward kernel: neighbour geometry
// and cutoffs (2 cap_a), `copies` copies of the float4 accumulators (one per
// neighbour each), a region that holds first the radial dE/dG (S * 16 <= 128
// floats) and then up to kGallBlocks angular blocks' dE/dG (9 float4s per block:
// 8 in feature order and one of padding, so that lanes reading float4 i of
// different blocks hit different banks), and the bytes of the neighbours' species and of
// the species-pair -> block-slot table (64)
constexpr int kGallStride = 9;
__host__ __device__ constexpr int aev_bwd_gall_f4(int n_pairs) {
  return kGallStride * (n_pairs < kGallBlocks ? n_pairs : kGallBlocks) > 32
             ? kGallStride * (n_pairs < kGallBlocks ? n_pairs : kGallBlocks)
             : 32;
}
__host__ __device__ constexpr int aev_bwd_warp_f4(int cap_a, int n_pairs, int copies) {
  return 2 * cap_a + copies * cap_a + aev_bwd_gall_f4(n_pairs) + (cap_a + 64 + 15) / 16;
}

// Copies of the per-neighbour angular accumulators.  The triplets are taken in
// round-robin order (rr_pair below): one round pairs every neighbour at most
// once, and the lanes of one 32-triplet pass span at most `copies` consecutive
// rounds, round r adding into copy r mod copies, so no two lanes of a pass add
// into the same accumulator and plain read-add-write is race-free.  4, 2 or 1:
// the most that keep four CTAs on an SM (228 KiB of shared memory per SM, 1 KiB
// reserved per CTA, plus the static list headers).
constexpr int kBwdCtaSmem = 228 * 1024 / 4 - 1024 - kWarps * (int)sizeof(ListHdr);
int aev_bwd_copies(int cap_a, int n_pairs) {
  for (int r = 4; r > 1; r >>= 1)
    if ((size_t)kWarps * aev_bwd_warp_f4(cap_a, n_pairs, r) * sizeof(float4) <= (size_t)kBwdCtaSmem)
      return r;
  return 1;
}

// The unordered pairs of n neighbours as rounds of disjoint pairs (the circle
// method of round-robin tournament scheduling).  n even: n - 1 rounds of
// h = n / 2 pairs, round r = (r, n - 1) and (r + i, r - i) mod (n - 1) for
// i = 1 .. h - 1; n odd: n rounds of h = (n - 1) / 2 pairs, (r + i, r - i) mod n
// for i = 1 .. h (neighbour r sits the round out).  Pair t is pair t mod h of
// round t / h; every unordered pair occurs once.
struct RoundRobin {
  int n, m, h, off, n_tri;   // m: the circle's size; off: 1 for odd n
  float inv_h;
};
__device__ __forceinline__ RoundRobin make_round_robin(int n) {
  RoundRobin rr;
  rr.n = n;
  const bool odd = n & 1;
  rr.m = odd ? n : n - 1;
  rr.h = max(odd ? (n - 1) / 2 : n / 2, 1);
  rr.off = odd ? 1 : 0;
  rr.n_tri = n * (n - 1) / 2;
  rr.inv_h = rcp_approx((float)rr.h);   // rr_round corrects the estimate by one step
  return rr;
}
// round of pair t (exact: the float estimate is corrected by one step)
__device__ __forceinline__ int rr_round(const RoundRobin& rr, int t) {
  int r = (int)((t + 0.5f) * rr.inv_h);
  if (r * rr.h > t) --r;
  else if ((r + 1) * rr.h <= t) ++r;
  return r;
}
__device__ __forceinline__ void rr_pair(const RoundRobin& rr, int t, int* round, int* a, int* b) {
  const int r = rr_round(rr, t);
  const int i = t - r * rr.h + rr.off;
  int x = r + i, y = r - i;
  if (x >= rr.m) x -= rr.m;
  if (y < 0) y += rr.m;
  if (i == 0) {   // even n: the fixed neighbour n - 1
    x = r;
    y = rr.n - 1;
  }
  *round = r;
  *a = x;
  *b = y;
}

__device__ __forceinline__ void load_hdr(const uint16_t* hdr, int S, unsigned lane, ListHdr* h) {
  int cr = (lane < (unsigned)S) ? hdr[lane] : 0;
  int ca = (lane < (unsigned)S) ? hdr[8 + lane] : 0;
  int ir = cr, ia = ca;
  for (int o = 1; o < 16; o <<= 1) {
    int u = __shfl_up_sync(kFull, ir, o);
    int v = __shfl_up_sync(kFull, ia, o);
    if ((int)lane >= o) { ir += u; ia += v; }
  }
  if (lane <= (unsigned)kMaxSpecies) {
    h->off_r[lane] = ir - cr;
    h->off_a[lane] = ia - ca;
  }
  __syncwarp();
}

// (j, k) of triplet t inside the block of species pair (s, u):
// same species: the t-th pair j < k of c atoms (row-major); else j = t / cu, k = t % cu
__device__ __forceinline__ void decode_pair(int t, int same, int c, int cu, float inv_cu,
                                            int* j, int* k) {
  if (same) {
    const float b = 2.f * c - 1.f;
    int jj = (int)((b - sqrt_approx(fmaxf(b * b - 8.f * t, 0.f))) * 0.5f);
    jj = max(0, min(jj, c - 2));
    if ((jj + 1) * (2 * c - jj - 2) / 2 <= t) ++jj;
    else if (jj * (2 * c - jj - 1) / 2 > t) --jj;
    *j = jj;
    *k = t - jj * (2 * c - jj - 1) / 2 + jj + 1;
  } else {
    int jj = (int)((t + 0.5f) * inv_cu);
    int kk = t - jj * cu;
    if (kk < 0) { --jj; kk += cu; }
    else if (kk >= cu) { ++jj; kk -= cu; }
    *j = jj;
    *k = kk;
  }
}

// Same pairs, numbered along diagonals so that consecutive lanes get distinct
// j (and distinct k): same species: pair (q, q + g + 1) of diagonal g; else
// d = t / cs, j = t % cs, k = (j + d) % cu.  Used where lanes add into
// per-neighbour accumulators, to spread those atomics over different addresses.
__device__ __forceinline__ void decode_pair_diag(int t, int same, int c, int cu, float inv_cs,
                                                 float inv_cu, int* j, int* k) {
  if (same) {
    const float b = 2.f * c - 1.f;
    int g = (int)((b - sqrt_approx(fmaxf(b * b - 8.f * t, 0.f))) * 0.5f);
    g = max(0, min(g, c - 2));
    if ((g + 1) * (2 * c - g - 2) / 2 <= t) ++g;
    else if (g * (2 * c - g - 1) / 2 > t) --g;
    const int q = t - g * (2 * c - g - 1) / 2;
    *j = q;
    *k = q + g + 1;
  } else {
    int d = (int)((t + 0.5f) * inv_cs);
    int jj = t - d * c;
    if (jj < 0) { --d; jj += c; }
    else if (jj >= c) { ++d; jj -= c; }
    const int x = jj + d;
    int kk = x - (int)((x + 0.5f) * inv_cu) * cu;
    if (kk < 0) kk += cu;
    else if (kk >= cu) kk -= cu;
    *j = jj;
    *k = kk;
  }
}

// one AEV element: the FP32 row, or on the tensor-core paths (Gh != null) only
// what their first layer reads: the BF16 row, and on the split path (Gl != null)
// also the low part bf16(v - bf16(v))
__device__ __forceinline__ void put_g(float* G, uint16_t* Gh, uint16_t* Gl, int f, float v) {
  if (Gh) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    Gh[f] = __bfloat16_as_ushort(h);
    if (Gl) Gl[f] = __bfloat16_as_ushort(__float2bfloat16_rn(v - __bfloat162float(h)));
  } else {
    G[f] = v;
  }
}

// after the call lane l holds the warp sum of v[l]
__device__ __forceinline__ float transpose_reduce32(float (&v)[32], unsigned lane) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool up = lane & o;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const float send = up ? v[i] : v[i + o];
      const float keep = up ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(kFull, send, o);
    }
  }
  return v[0];
}

// The 64-column slices of a centre's AEV row that hold a block with any term:
// radial block s (columns 16 s ..) when the centre has neighbours of species s,
// angular block q of species pair (s, u) (columns 16 S + 32 q ..) when it has a
// pair j < k of those species; bit 0 is always set.  All other slices of the row
// are zero.  The same value on every lane.
// pair_su[q] = s | u << 4 for species pair q (s <= u, upper triangle row-major)
__device__ __forceinline__ void fill_pair_table(uint8_t* pair_su, const AevConst& ac) {
  for (int q = threadIdx.x; q < ac.n_pairs; q += blockDim.x) {
    int sp = 0, rem = q;
    while (rem >= ac.S - sp) { rem -= ac.S - sp; ++sp; }
    pair_su[q] = (uint8_t)(sp | ((sp + rem) << 4));
  }
}

__device__ __forceinline__ uint32_t row_slices(const ListHdr& H, const AevConst& ac, unsigned lane,
                                               const uint8_t* pair_su) {
  uint32_t m = 1u;
  if ((int)lane < ac.S && H.off_r[lane + 1] > H.off_r[lane]) m |= 1u << (ac.rcol[lane] >> 6);
  for (int q = (int)lane; q < ac.n_pairs; q += 32) {
    const int sp = pair_su[q] & 15, u = pair_su[q] >> 4;
    const int cs = H.off_a[sp + 1] - H.off_a[sp], cu = H.off_a[u + 1] - H.off_a[u];
    if (sp == u ? cs >= 2 : (cs > 0 && cu > 0)) {
      const int f0 = ac.acol[q];
      m |= (1u << (f0 >> 6)) | (1u << ((f0 + 31) >> 6));
    }
  }
  return __reduce_or_sync(kFull, m);
}

// whether a block of `width` columns from f0 touches a slice of mask m
__device__ __forceinline__ bool block_in(uint32_t m, int f0, int width) {
  const int a = f0 >> 6, b = (f0 + width - 1) >> 6;
  return (m >> a) & 1u || (m >> b) & 1u;
}

// float4s of per-warp shared memory of the forward: angular unit vectors and R
// (cap_a), angular cutoffs (cap_a floats + 4), radial (R, f_c) pairs (cap_r)
__host__ __device__ constexpr int aev_fwd_warp_f4(int cap_a, int cap_r) {
  return cap_a + cap_a / 4 + cap_r / 2 + 2;
}

// The AEV row of packed atom p (Eqs. 3-5) by one warp; out(f, v) stores feature
// f (each f < Dp exactly once, by the lane holding it).  stage: this warp's
// aev_fwd_warp_f4 float4s of shared memory; H: its list header.  With sparse
// set, only the blocks that touch a live slice of the row (row_slices) are
// stored, and *mask receives the row's slice mask.
template <int ZETA, class Out>
__device__ __forceinline__ void aev_centre(const Ws& ws, const AevConst& ac, int p, float4* stage,
                                           ListHdr& H, unsigned lane, const uint8_t* pair_su,
                                           Out out, bool sparse = false, uint32_t* mask = nullptr) {
  __syncwarp();   // the warp's stage and header may still hold its previous centre
  float4* angv = stage;
  float* angf = reinterpret_cast<float*>(angv + ws.cap_a);
  float2* rad = reinterpret_cast<float2*>(angf + ws.cap_a + 4);
  const float4 xi = ws.xyzq[p];
  const SysDev& d = ws.sys[ws.pos_sys[p]];
  {   // the first lines of the neighbour lists travel while the header loads
    const int* a = nullptr;
    if (lane < 2 && (int)lane * 32 < ws.cap_r) a = ws.nb_r + (size_t)p * ws.cap_r + lane * 32;
    else if (lane == 2) a = ws.nb_a + (size_t)p * ws.cap_a;
    if (a) asm volatile("prefetch.global.L1 [%0];" ::"l"(a));
  }
  load_hdr(ws.nb_cnt + (size_t)p * 16, ac.S, lane, &H);
  const uint32_t m = sparse ? row_slices(H, ac, lane, pair_su) : ~0u;
  if (mask) *mask = m;
  const int* lr = ws.nb_r + (size_t)p * ws.cap_r;
  const int* la = ws.nb_a + (size_t)p * ws.cap_a;
  const float inv_rc_r = 1.f / ac.rc_r, inv_rc_a = 1.f / ac.rc_a;
  stage_list(H.off_r[ac.S], lr, xi, d, ws, lane,
             [&](int slot, int, const Geo& g) {
               rad[slot] = make_float2(g.r, fcut(g.r, ac.rc_r, inv_rc_r));
             });
  stage_list(H.off_a[ac.S], la, xi, d, ws, lane,
             [&](int slot, int, const Geo& g) {
               const float inv = rcp_approx(g.r);
               angv[slot] = make_float4(g.dx * inv, g.dy * inv, g.dz * inv, g.r);
               angf[slot] = fcut(g.r, ac.rc_a, inv_rc_a);
             });
  __syncwarp();
  // ---- radial, Eq. 4
  const float cr_ = -ac.eta_r * kLog2e;
  const float my_shf = ac.shf_r[lane & 15];
  const int half = lane >> 4;
  for (int s = 0; s < ac.S; ++s) {
    float acc = 0.f;
    const int o = H.off_r[s], n = H.off_r[s + 1] - o;
    if (n == 0) {   // no neighbour of this species: a zero block
      if (lane < 16 && block_in(m, ac.rcol[s], kNR)) out(ac.rcol[s] + lane, 0.f);
      continue;
    }
    for (int t = half; t < n; t += 2) {
      const float2 q = rad[o + t];
      const float x = q.x - my_shf;
      acc = fmaf(fast_exp2(cr_ * x * x), q.y, acc);
    }
    acc += __shfl_xor_sync(kFull, acc, 16);
    if (lane < 16 && block_in(m, ac.rcol[s], kNR)) out(ac.rcol[s] + lane, acc);
  }
  // ---- angular, Eq. 5: the blocks of species pairs with a pair j < k, and the
  // zero blocks of the other pairs where the row is written
  const float ca_ = -ac.eta_a * kLog2e;
  uint32_t live[2] = {0u, 0u}, zero[2] = {0u, 0u};
  for (int h = 0; h * 32 < ac.n_pairs; ++h) {
    const int q = h * 32 + (int)lane;
    bool lv = false, zr = false;
    if (q < ac.n_pairs) {
      const int sp = pair_su[q] & 15, u = pair_su[q] >> 4;
      const int cs = H.off_a[sp + 1] - H.off_a[sp], cu = H.off_a[u + 1] - H.off_a[u];
      lv = sp == u ? cs >= 2 : (cs > 0 && cu > 0);
      zr = !lv && block_in(m, ac.acol[q], 32);
    }
    live[h] = __ballot_sync(kFull, lv);
    zero[h] = __ballot_sync(kFull, zr);
  }
  for (int h = 0; h < 2; ++h)
    for (uint32_t z = zero[h]; z; z &= z - 1)
      out(ac.acol[h * 32 + __ffs(z) - 1] + lane, 0.f);
  for (int h = 0; h < 2; ++h)
    for (uint32_t lv = live[h]; lv; lv &= lv - 1) {
      const int q = h * 32 + __ffs(lv) - 1;
      const int s = pair_su[q] & 15, u = pair_su[q] >> 4;
      const int os = H.off_a[s], cs = H.off_a[s + 1] - os;
      const int ou = H.off_a[u], cu = H.off_a[u + 1] - ou;
      const int same = (s == u);
      const int n_tri = same ? cs * (cs - 1) / 2 : cs * cu;
      const int fb = ac.acol[q];
      const float inv_cu = rcp_approx((float)max(cu, 1));   // decode corrects one step either way
      // acc2[4a + m] holds features 8a + 2m and 8a + 2m + 1 (packed FP32x2 FMAs)
      float2 acc2[16];
#pragma unroll
      for (int f = 0; f < 16; ++f) acc2[f] = make_float2(0.f, 0.f);
      for (int t0 = 0; t0 < n_tri; t0 += 32) {
        const int t = t0 + lane;
        if (t < n_tri) {
          int j, k;
          decode_pair(t, same, cs, cu, inv_cu, &j, &k);
          const float4 vj = angv[os + j];
          const float4 vk = angv[ou + k];
          const float fjk = ac.ang_pre * angf[os + j] * angf[ou + k];
          const float chat = vj.x * vk.x + vj.y * vk.y + vj.z * vk.z;
          const float c = ac.cos_scale * chat;
          const float sn = sin_theta(vj, vk, chat, ac.cos_scale);
          const float rb = 0.5f * (vj.w + vk.w);
          float2 A[kNA];
#pragma unroll
          for (int a = 0; a < kNA; ++a) {
            const float x = rb - ac.shf_a[a];
            const float v = fast_exp2(ca_ * x * x) * fjk;
            A[a] = make_float2(v, v);
          }
          const float2 c2 = make_float2(c, c), s2 = make_float2(sn, sn);
#pragma unroll
          for (int m = 0; m < kNZ / 2; ++m) {
            const float2 B = section_pair<ZETA>(ac, m, c2, s2);
#pragma unroll
            for (int a = 0; a < kNA; ++a) acc2[4 * a + m] = __ffma2_rn(A[a], B, acc2[4 * a + m]);
          }
        }
      }
      float acc[32];
#pragma unroll
      for (int f = 0; f < 16; ++f) {
        acc[2 * f] = acc2[f].x;
        acc[2 * f + 1] = acc2[f].y;
      }
      out(fb + lane, transpose_reduce32(acc, lane));
    }
  for (int f = ac.D + lane; f < ac.Dp; f += 32)
    if ((m >> (f >> 6)) & 1u) out(f, 0.f);
}

template <int ZETA>
__global__ void __launch_bounds__(kWarps * 32, 4)
k_aev_fwd(Ws ws, AevConst ac) {
  extern __shared__ float4 sm4[];
  __shared__ ListHdr hdrs[kWarps];
  __shared__ uint8_t pair_su[kMaxSpecies * (kMaxSpecies + 1) / 2];
  const int w = threadIdx.x >> 5;
  const unsigned lane = threadIdx.x & 31;
  const bool sparse = ws.row_mask != nullptr;
  fill_pair_table(pair_su, ac);
  __syncthreads();
  // persistent: every warp takes the next centre from a counter until none is left
  // (dense centres do not hold a CTA's other warps' slots, nor pile up in one warp)
  const int n = ws.totals[0];
  for (;;) {
    int p = 0;
    if (lane == 0) p = atomicAdd(ws.totals + 4, 1);
    p = __shfl_sync(kFull, p, 0);
    if (p >= n) break;
    if (!NNP_IN_BOUNDS(ws.status, kSiteAevRow, ws.pos_slot[p], ws.row_cap)) continue;
    const size_t row = (size_t)ws.pos_slot[p] * ac.Dp;
    float* G = ws.aev + row;
    uint16_t* Gh = ws.aev_h ? ws.aev_h + row : nullptr;
    uint16_t* Gl = ws.aev_l ? ws.aev_l + row : nullptr;
    uint32_t m = 0;
    aev_centre<ZETA>(ws, ac, p, sm4 + (size_t)w * aev_fwd_warp_f4(ws.cap_a, ws.cap_r), hdrs[w], lane,
                     pair_su, [&](int f, float v) { put_g(G, Gh, Gl, f, v); }, sparse, &m);
    if (sparse && lane == 0) {
      const int slot = ws.pos_slot[p];
      ws.row_mask[slot] = m;
      atomicOr(ws.tile_mask + (slot >> 7), m);
    }
  }
}

// One warp per AEV row of a species segment: zero the 64-column slices the row's
// tile reads (tile mask) that the row did not write (row mask).  Padding rows
// past a segment's atoms are left alone (their network outputs are never read).
__global__ void __launch_bounds__(256) k_aev_fill(Ws ws, AevConst ac) {
  const int r = blockIdx.x * 8 + (threadIdx.x >> 5);
  const unsigned lane = threadIdx.x & 31;
  if (r >= ws.seg_start[ac.S]) return;
  int s = 0;
  while (s + 1 < ac.S && r >= ws.seg_start[s + 1]) ++s;
  if (r >= ws.seg_start[s] + ws.species_count[s]) return;
  uint32_t miss = ws.tile_mask[r >> 7] & ~ws.row_mask[r];
  const size_t row = (size_t)r * ac.Dp;
  while (miss) {
    const int k = __ffs(miss) - 1;
    miss &= miss - 1;
    const int f = k * 64 + 2 * (int)lane;      // two columns per lane
    if (f < ac.Dp) {
      reinterpret_cast<uint32_t*>(ws.aev_h + row + f)[0] = 0u;
      if (ws.aev_l) reinterpret_cast<uint32_t*>(ws.aev_l + row + f)[0] = 0u;
    }
  }
}

// ---- backward pieces shared by the warp-per-centre and CTA-per-centre kernels

// One radial edge (Eq. 4) of centre i: dE/dr_ij from the S*16 radial dE/dG
// values gs of neighbour j's species; the force on j goes to f_pos[j] at once,
// the centre's share (and the virial) into the caller's accumulators.
template <bool VIR>
__device__ __forceinline__ void radial_edge_bwd(const Ws& ws, const AevConst& ac, const float4& xi,
                                                const SysDev& d, int j, const float4& xj,
                                                const float* gs, float inv_rc_r, float* fi,
                                                float* vir, float4* det_slot) {
  const float cr_ = -ac.eta_r * kLog2e;
  const Geo g = pair_geo(xi, xj, d);
  float fc, dfc;
  fcut_both(g.r, ac.rc_r, inv_rc_r, &fc, &dfc);
  // dE/dR = sum_r g_r e_r (-2 eta x_r f_c + f_c') = f_c (-2 eta) sum_r g_r e_r x_r + f_c' sum_r g_r e_r
  // (shells in pairs: packed FP32x2 arithmetic, sums over the even and odd shells)
  const float2 r2 = make_float2(g.r, g.r), cr2 = make_float2(cr_, cr_);
  const float2* shf2 = reinterpret_cast<const float2*>(ac.shf_r);
  const float2* gs2 = reinterpret_cast<const float2*>(gs);   // gs: 8-byte aligned
  float2 sge2 = make_float2(0.f, 0.f), sgex2 = make_float2(0.f, 0.f);
#pragma unroll
  for (int m = 0; m < kNR / 2; ++m) {
    const float2 x = __ffma2_rn(shf2[m], make_float2(-1.f, -1.f), r2);
    const float2 q = __fmul2_rn(__fmul2_rn(x, x), cr2);
    const float2 ge = __fmul2_rn(gs2[m], make_float2(fast_exp2(q.x), fast_exp2(q.y)));
    sge2 = __fadd2_rn(sge2, ge);
    sgex2 = __ffma2_rn(ge, x, sgex2);
  }
  const float sge = sge2.x + sge2.y, sgex = sgex2.x + sgex2.y;
  const float dEdR = fmaf(fc * (-2.f * ac.eta_r), sgex, dfc * sge);
  const float sc = dEdR * rcp_approx(g.r);
  const float gx = sc * g.dx, gy = sc * g.dy, gz = sc * g.dz;
  if (det_slot) *det_slot = make_float4(-gx, -gy, -gz, 0.f);   // deterministic mode
  else atomicAdd(&ws.f_pos[j], make_float4(-gx, -gy, -gz, 0.f));
  fi[0] += gx; fi[1] += gy; fi[2] += gz;
  if (VIR) {
    vir[0] -= g.dx * gx; vir[1] -= g.dx * gy; vir[2] -= g.dx * gz;
    vir[3] -= g.dy * gx; vir[4] -= g.dy * gy; vir[5] -= g.dy * gz;
    vir[6] -= g.dz * gx; vir[7] -= g.dz * gy; vir[8] -= g.dz * gz;
  }
}

// Block table of a centre's angular terms, built by one warp: per species pair
// q, its geometry (os, cs, ou, cu | same << 16) in the species-sorted angular
// list and the number of its first triplet in a numbering continuous over all
// blocks (bt_start[n_pairs] = the centre's triplet count).
__device__ __forceinline__ void build_block_table(const ListHdr& H, const AevConst& ac,
                                                  unsigned lane, int4* bt_geo, int* bt_start) {
  const int np = ac.n_pairs;
  for (int q0 = 0, carry = 0; q0 < np; q0 += 32) {
    const int q = q0 + lane;
    int n_tri = 0;
    if (q < np) {
      int sp = 0, rem = q;
      while (rem >= ac.S - sp) { rem -= ac.S - sp; ++sp; }
      const int u = sp + rem;
      const int os = H.off_a[sp], cs = H.off_a[sp + 1] - os;
      const int ou = H.off_a[u], cu = H.off_a[u + 1] - ou;
      const int same = (sp == u);
      n_tri = same ? cs * (cs - 1) / 2 : cs * cu;
      bt_geo[q] = make_int4(os, cs, ou, cu | (same << 16));
    }
    int incl = n_tri;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(kFull, incl, o);
      if ((int)lane >= o) incl += v;
    }
    if (q < np) bt_start[q] = carry + incl - n_tri;
    carry += __shfl_sync(kFull, incl, 31);
    if (q0 + 32 >= np && lane == 0) bt_start[np] = carry;
  }
}

// One angular triplet (Eq. 5) of a centre: neighbours j and k (unit vector and
// R; f_c, f_c', 1/R), the 32 dE/dG values of their species-pair block in
// feature order (index 8a + z: float4 2a + h holds sections 4h .. 4h + 3 of
// radial shell a).  Returns dE/d(r_j) and dE/d(r_k) (the force terms on j and
// k; their negatives act on the centre).
template <int ZETA>
__device__ __forceinline__ void triplet_bwd(const AevConst& ac, const float4& vj, const float4& vk,
                                            const float4& fj4, const float4& fk4,
                                            const float4* gblk, float3& uj, float3& uk) {
  const float ca_ = -ac.eta_a * kLog2e;
  const float m2eta = -2.f * ac.eta_a;
  const float chat = vj.x * vk.x + vj.y * vk.y + vj.z * vk.z;
  const float c = ac.cos_scale * chat;
  const float sn = fmaxf(sin_theta(vj, vk, chat, ac.cos_scale), 1e-6f);
  const float m_c_over_s = -c * rcp_approx(sn);
  const float rb = 0.5f * (vj.w + vk.w);
  // contract the block's dE/dG over the 8 angle sections first:
  //   F_a = sum_z g[a][z] B_z,  dF_a = sum_z g[a][z] dB_z/dc,
  // dB_z/dc = zeta base^(zeta-1) (cos(theta_z) - sin(theta_z) c / s) (the factor
  // zeta is applied at the end); sections in pairs, Fp[a] holding the sums over
  // the even and the odd sections
  const float2 c2 = make_float2(c, c), s2 = make_float2(sn, sn);
  const float2 mcs2 = make_float2(m_c_over_s, m_c_over_s);
  float2 Fp[kNA], dFp[kNA];
#pragma unroll
  for (int a = 0; a < kNA; ++a) Fp[a] = dFp[a] = make_float2(0.f, 0.f);
  const float2* g2 = reinterpret_cast<const float2*>(gblk);
#pragma unroll
  for (int m = 0; m < kNZ / 2; ++m) {
    float2 B1;
    const float2 B = section_pair<ZETA>(ac, m, c2, s2, &B1);
    const float2 cz = reinterpret_cast<const float2*>(ac.cos_z)[m];
    const float2 sz = reinterpret_cast<const float2*>(ac.sin_z)[m];
    const float2 dB = __fmul2_rn(B1, __ffma2_rn(sz, mcs2, cz));
#pragma unroll
    for (int a = 0; a < kNA; ++a) {
      const float2 g = g2[4 * a + m];
      Fp[a] = __ffma2_rn(g, B, Fp[a]);
      dFp[a] = __ffma2_rn(g, dB, dFp[a]);
    }
  }
  float F[kNA], dF[kNA];
#pragma unroll
  for (int a = 0; a < kNA; ++a) {
    F[a] = Fp[a].x + Fp[a].y;
    dF[a] = dFp[a].x + dFp[a].y;
  }
  float tc = 0.f, tR = 0.f, tf = 0.f;
#pragma unroll
  for (int a = 0; a < kNA; ++a) {
    const float x = rb - ac.shf_a[a];
    const float A = fast_exp2(ca_ * x * x);
    const float AF = A * F[a];
    tf += AF;
    tR = fmaf(m2eta * x, AF, tR);
    tc = fmaf(A, dF[a], tc);
  }
  const float fjk = fj4.x * fk4.x;
  tc *= ac.ang_pre * (float)ac.zeta * fjk;  // dE/dc, c = cos_scale * cos_hat
  tR *= ac.ang_pre * fjk;                    // dE/dRbar
  tf *= ac.ang_pre;                          // dE/d(f_j f_k)
  const float dEdchat = ac.cos_scale * tc;
  const float sj = dEdchat * fj4.z, sk = dEdchat * fk4.z;
  const float rj = 0.5f * tR + tf * fj4.y * fk4.x;
  const float rk = 0.5f * tR + tf * fj4.x * fk4.y;
  uj = make_float3(sj * (vk.x - chat * vj.x) + rj * vj.x, sj * (vk.y - chat * vj.y) + rj * vj.y,
                   sj * (vk.z - chat * vj.z) + rj * vj.z);
  uk = make_float3(sk * (vj.x - chat * vk.x) + rk * vk.x, sk * (vj.y - chat * vk.y) + rk * vk.y,
                   sk * (vj.z - chat * vk.z) + rk * vk.z);
}

// Warp per centre, for centres with at most cap_l angular neighbours whose
// angular terms fall in at most kGallBlocks species-pair blocks (the blocks'
// dE/dG are all staged at once); a centre with more is appended to ws.heavy
// (count in totals[2]) for k_aev_bwd_heavy and skipped.
template <int ZETA, bool VIR>
__device__ __forceinline__ void bwd_centre(const Ws& ws, const AevConst& ac, int log_r, int cap_l,
                                           int p, float4* sm4, ListHdr& H, int w, unsigned lane) {
  __syncwarp();   // the warp's previous centre is done with its shared memory
  const bool det = ws.fr_det != nullptr;   // deterministic mode
  const int n_copy = 1 << log_r;
  float4* angv = sm4 + (size_t)w * aev_bwd_warp_f4(cap_l, ac.n_pairs, n_copy);
  float4* angf = angv + cap_l;             // fc, dfc, 1/R, packed index
  float4* acc = angf + cap_l;              // dE/du per neighbour, [copy][neighbour]
  float4* uni = acc + (size_t)n_copy * cap_l;
  float* grad = reinterpret_cast<float*>(uni);   // S*16 radial dE/dG, then:
  float4* gall = uni;                            // angular dE/dG, [slot][8a + z] (+ pad)
  uint8_t* spec = reinterpret_cast<uint8_t*>(uni + aev_bwd_gall_f4(ac.n_pairs));  // [cap_l]
  uint8_t* pslot = spec + cap_l;           // [8 s + u]: block slot of species pair (s, u)

  const float4 xi = ws.xyzq[p];
  const SysDev& d = ws.sys[ws.pos_sys[p]];
  const float* g_row = ws.dEdG + (size_t)ws.pos_slot[p] * ac.Dp;
  load_hdr(ws.nb_cnt + (size_t)p * 16, ac.S, lane, &H);
  // species-pair blocks with triplets: pairs of present species and species
  // present at least twice
  int n_live;
  {
    const int c = (int)lane < ac.S ? H.off_a[lane + 1] - H.off_a[lane] : 0;
    const int n_one = __popc(__ballot_sync(kFull, c >= 1));
    const int n_two = __popc(__ballot_sync(kFull, c >= 2));
    n_live = n_one * (n_one - 1) / 2 + n_two;
  }
  if (H.off_a[ac.S] > cap_l || n_live > kGallBlocks) {
    if (lane == 0) {
      const int hi = atomicAdd(ws.totals + 2, 1);
      if (NNP_IN_BOUNDS(ws.status, kSiteBwdHeavy, hi, ws.n_in)) ws.heavy[hi] = p;
    }
    return;
  }
  const int* lr = ws.nb_r + (size_t)p * ws.cap_r;
  const int* la = ws.nb_a + (size_t)p * ws.cap_a;
  const float inv_rc_r = 1.f / ac.rc_r, inv_rc_a = 1.f / ac.rc_a;
  // the radial dE/dG (S * 16 <= 128 values) is loaded now and stored after the
  // neighbour gathers, so that the two latencies overlap
  float gr[kMaxSpecies * kNR / 32];
#pragma unroll
  for (int i = 0; i < kMaxSpecies * kNR / 32; ++i) {
    const int f = (int)lane + 32 * i;
    gr[i] = f < ac.S * kNR ? g_row[ac.rcol[f >> 4] + (f & 15)] : 0.f;
  }
  // angular neighbours: unit vector and R, (f_c, f_c', 1/R, packed index), species
  stage_list(H.off_a[ac.S], la, xi, d, ws, lane,
             [&](int slot, int j, const Geo& g) {
               const float inv = rcp_approx(g.r);
               angv[slot] = make_float4(g.dx * inv, g.dy * inv, g.dz * inv, g.r);
               float fc, dfc;
               fcut_both(g.r, ac.rc_a, inv_rc_a, &fc, &dfc);
               angf[slot] = make_float4(fc, dfc, inv, __int_as_float(j));
             });
  const int na_tot = H.off_a[ac.S];
  for (int t = lane; t < na_tot; t += 32) {
    int s = 0;
    while (s + 1 < ac.S && H.off_a[s + 1] <= t) ++s;
    spec[t] = (uint8_t)s;
  }
  for (int c = 0; c < n_copy; ++c)
    for (int t = lane; t < na_tot; t += 32) acc[c * cap_l + t] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int i = 0; i < kMaxSpecies * kNR / 32; ++i) {
    const int f = (int)lane + 32 * i;
    if (f < ac.S * kNR) grad[f] = gr[i];
  }
  __syncwarp();
  float fi[3] = {0.f, 0.f, 0.f};
  float vir[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) vir[k] = 0.f;
  // ---- radial edges, one lane per neighbour, numbered continuously over the
  // species blocks of the list (a lane finds its neighbour's species block);
  // two neighbours per lane and pass, both gathers issued before either is used
  const int nr_tot = H.off_r[ac.S];
  int sr = 0;
  for (int t0 = 0; t0 < nr_tot; t0 += 64) {
    const int ta = t0 + (int)lane, tb = ta + 32;
    int ja = ta < nr_tot ? lr[ta] : -1;
    int jb = tb < nr_tot ? lr[tb] : -1;
    if (ja >= 0 && !NNP_IN_BOUNDS(ws.status, kSiteBwdNeighbour, ja, ws.totals[0])) ja = -1;
    if (jb >= 0 && !NNP_IN_BOUNDS(ws.status, kSiteBwdNeighbour, jb, ws.totals[0])) jb = -1;
    const float4 xa = ja >= 0 ? ws.xyzq[ja] : xi;
    const float4 xb = jb >= 0 ? ws.xyzq[jb] : xi;
    if (ja >= 0) {
      while (H.off_r[sr + 1] <= ta) ++sr;
      radial_edge_bwd<VIR>(ws, ac, xi, d, ja, xa, grad + sr * kNR, inv_rc_r, fi, vir,
                           det ? ws.fr_det + (size_t)p * ws.cap_r + ta : nullptr);
    }
    if (jb >= 0) {
      while (H.off_r[sr + 1] <= tb) ++sr;
      radial_edge_bwd<VIR>(ws, ac, xi, d, jb, xb, grad + sr * kNR, inv_rc_r, fi, vir,
                           det ? ws.fr_det + (size_t)p * ws.cap_r + tb : nullptr);
    }
  }
  __syncwarp();   // the radial dE/dG's region now takes the angular blocks
  // ---- the live species-pair blocks: slot k of the k-th live pair (s <= u) in
  // the order 8 s + u, its dE/dG (32 values, index 8a + z) staged in that order
  {
    float* gf = reinterpret_cast<float*>(gall);
    unsigned m[2];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int l = 32 * half + (int)lane, s = l >> 3, u = l & 7;
      bool live = false;
      if (s <= u && u < ac.S) {
        const int cs = H.off_a[s + 1] - H.off_a[s], cu = H.off_a[u + 1] - H.off_a[u];
        live = s == u ? cs >= 2 : (cs >= 1 && cu >= 1);
      }
      m[half] = __ballot_sync(kFull, live);
      if (live) {
        const int slot = (half ? __popc(m[0]) : 0) + __popc(m[half] & ((1u << lane) - 1u));
        pslot[8 * s + u] = (uint8_t)slot;
        pslot[8 * u + s] = (uint8_t)slot;
      }
    }
    // the blocks' loads are issued four at a time before their stores
    for (int k0 = 0; k0 < n_live; k0 += 4) {
      float gv[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        gv[k] = 0.f;
        if (k0 + k < n_live) {
          int l;
          if (m[0]) { l = __ffs(m[0]) - 1; m[0] &= m[0] - 1; }
          else { l = 32 + __ffs(m[1]) - 1; m[1] &= m[1] - 1; }
          const int s = l >> 3, u = l & 7;
          const int q = s * ac.S - s * (s - 1) / 2 + (u - s);
          gv[k] = g_row[ac.acol[q] + lane];
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k0 + k < n_live) gf[(k0 + k) * (4 * kGallStride) + lane] = gv[k];
    }
  }
  __syncwarp();
  // ---- angular triplets in round-robin order, one lane per pair: a pass takes
  // the next 32 pairs but at most n_copy rounds, round r adding into copy
  // r mod n_copy with plain read-add-write (within a round the pairs are
  // disjoint, so no two lanes of a pass touch the same accumulator); the order
  // of every addition is fixed, in the deterministic mode too
  const RoundRobin rr = make_round_robin(na_tot);
  for (int t0 = 0; t0 < rr.n_tri;) {
    const int r0 = rr_round(rr, t0);
    const int t1 = min(min(t0 + 32, (r0 + n_copy) * rr.h), rr.n_tri);
    const int t = t0 + (int)lane;
    if (t < t1) {
      int r, a, b;
      rr_pair(rr, t, &r, &a, &b);
      if (NNP_IN_BOUNDS(ws.status, kSiteBwdTriplet, a, na_tot) &&
          NNP_IN_BOUNDS(ws.status, kSiteBwdTriplet, b, na_tot)) {
        const int slot = pslot[8 * spec[a] + spec[b]];
        if (NNP_IN_BOUNDS(ws.status, kSiteBwdTriplet, slot, n_live)) {
          float3 ua, ub;
          triplet_bwd<ZETA>(ac, angv[a], angv[b], angf[a], angf[b], gall + slot * kGallStride,
                            ua, ub);
          float4* A = acc + (r & (n_copy - 1)) * cap_l;
          float4 x = A[a];
          x.x += ua.x; x.y += ua.y; x.z += ua.z;
          A[a] = x;
          float4 y = A[b];
          y.x += ub.x; y.y += ub.y; y.z += ub.z;
          A[b] = y;
        }
      }
    }
    __syncwarp();   // the next pass may add into the same accumulators
    t0 = t1;
  }
  for (int t = lane; t < na_tot; t += 32) {
    float4 a = acc[t];
    for (int c = 1; c < n_copy; ++c) {
      const float4 v = acc[c * cap_l + t];
      a.x += v.x;
      a.y += v.y;
      a.z += v.z;
    }
    const float4 v = angv[t];
    const int jt = __float_as_int(angf[t].w);
    if (det) ws.fa_det[(size_t)p * ws.cap_a + t] = make_float4(-a.x, -a.y, -a.z, 0.f);
    else if (NNP_IN_BOUNDS(ws.status, kSiteBwdNeighbour, jt, ws.totals[0]))
      atomicAdd(&ws.f_pos[jt], make_float4(-a.x, -a.y, -a.z, 0.f));
    fi[0] += a.x; fi[1] += a.y; fi[2] += a.z;
    if (VIR) {
      const float ux = v.x * v.w, uy = v.y * v.w, uz = v.z * v.w;
      vir[0] -= ux * a.x; vir[1] -= ux * a.y; vir[2] -= ux * a.z;
      vir[3] -= uy * a.x; vir[4] -= uy * a.y; vir[5] -= uy * a.z;
      vir[6] -= uz * a.x; vir[7] -= uz * a.y; vir[8] -= uz * a.z;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fi[0] += __shfl_xor_sync(kFull, fi[0], o);
    fi[1] += __shfl_xor_sync(kFull, fi[1], o);
    fi[2] += __shfl_xor_sync(kFull, fi[2], o);
  }
  if (lane == 0) {
    if (det) ws.fs_det[p] = make_float4(fi[0], fi[1], fi[2], 0.f);
    else atomicAdd(&ws.f_pos[p], make_float4(fi[0], fi[1], fi[2], 0.f));
  }
  if (VIR && d.in.virial) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      float v = vir[k];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
      if (lane == 0) {
        if (det) ws.v_det[(size_t)p * 9 + k] = (double)v;
        else atomicAdd(d.in.virial + k, (double)v);
      }
    }
  }
}

template <int ZETA, bool VIR>
__global__ void __launch_bounds__(kWarps * 32, 4)
k_aev_bwd(Ws ws, AevConst ac, int log_r, int cap_l) {
  extern __shared__ float4 sm4[];
  __shared__ ListHdr hdrs[kWarps];
  const int w = threadIdx.x >> 5;
  const unsigned lane = threadIdx.x & 31;
  // persistent: every warp takes the next centre from a counter until none is left
  const int n = ws.totals[0];
  for (;;) {
    int p = 0;
    if (lane == 0) p = atomicAdd(ws.totals + 5, 1);
    p = __shfl_sync(kFull, p, 0);
    if (p >= n) break;
    bwd_centre<ZETA, VIR>(ws, ac, log_r, cap_l, p, sm4, hdrs[w], w, lane);
  }
}

// CTA per centre, for the centres k_aev_bwd handed on (more than its cap_l
// angular neighbours: a dense solute core can have a hundred, i.e. thousands of
// triplets).  The CTA's eight warps share the centre's staged neighbours and all
// its angular dE/dG blocks and split its radial edges and triplets; every warp
// adds into its own copies of the per-neighbour accumulators (lane l into copy
// (l mod n_lane) of its warp's n_lane), summed once at the end.  Persistent:
// CTAs stride over the ws.heavy list.
constexpr int kHeavyThreads = 256;

__host__ __device__ constexpr size_t aev_bwd_heavy_smem(int cap_a, int n_pairs, int n_lane) {
  return (size_t)2 * cap_a * 16 +                        // angv, angf
         (size_t)3 * cap_a * (kHeavyThreads / 32) * n_lane * 4 +  // accumulators
         (size_t)kMaxSpecies * kNR * 4 +                  // radial dE/dG
         (size_t)n_pairs * 32 * 4 +                       // angular dE/dG, [q][8a + z]
         (size_t)n_pairs * 16 + (size_t)(n_pairs + 1) * 4 + 16;   // block table
}

template <int ZETA, bool VIR>
__global__ void __launch_bounds__(kHeavyThreads)
k_aev_bwd_heavy(Ws ws, AevConst ac, int log_n) {
  extern __shared__ float4 smh[];
  __shared__ ListHdr H;
  __shared__ float red[kHeavyThreads / 32][12];
  const int n_lane = 1 << log_n;
  const int n_acc = (kHeavyThreads / 32) << log_n;      // copies per neighbour
  const int cap = ws.cap_a;
  const int tid = threadIdx.x, w = tid >> 5;
  const unsigned lane = tid & 31;
  float4* angv = smh;
  float4* angf = angv + cap;
  float* accx = reinterpret_cast<float*>(angf + cap);   // [neighbour][copy]
  float* accy = accx + (size_t)cap * n_acc;
  float* accz = accy + (size_t)cap * n_acc;
  float* grad = accz + (size_t)cap * n_acc;
  float* gf = grad + kMaxSpecies * kNR;
  const float4* gall = reinterpret_cast<const float4*>(gf);
  int4* bt_geo = reinterpret_cast<int4*>(gf + ac.n_pairs * 32);
  int* bt_start = reinterpret_cast<int*>(bt_geo + ac.n_pairs);
  const int np = ac.n_pairs;
  const int n_heavy = ws.totals[2];
  const bool det = ws.fr_det != nullptr;   // deterministic mode
  const float inv_rc_r = 1.f / ac.rc_r, inv_rc_a = 1.f / ac.rc_a;
  for (int h = blockIdx.x; h < n_heavy; h += gridDim.x) {
    const int p = ws.heavy[h];
    __syncthreads();   // the previous centre's shared data are no longer read
    if (w == 0) load_hdr(ws.nb_cnt + (size_t)p * 16, ac.S, lane, &H);
    __syncthreads();
    const float4 xi = ws.xyzq[p];
    const SysDev& d = ws.sys[ws.pos_sys[p]];
    const float* g_row = ws.dEdG + (size_t)ws.pos_slot[p] * ac.Dp;
    const int* lr = ws.nb_r + (size_t)p * ws.cap_r;
    const int* la = ws.nb_a + (size_t)p * ws.cap_a;
    const int na = H.off_a[ac.S], nr = H.off_r[ac.S];
    for (int t = tid; t < na; t += kHeavyThreads) {
      int j = la[t];
      if (!NNP_IN_BOUNDS(ws.status, kSiteAevNeighbour, j, ws.totals[0])) j = p;
      const Geo g = pair_geo(xi, ws.xyzq[j], d);
      const float inv = rcp_approx(g.r);
      angv[t] = make_float4(g.dx * inv, g.dy * inv, g.dz * inv, g.r);
      float fc, dfc;
      fcut_both(g.r, ac.rc_a, inv_rc_a, &fc, &dfc);
      angf[t] = make_float4(fc, dfc, inv, __int_as_float(j));
    }
    for (int i = tid; i < na * n_acc; i += kHeavyThreads) {
      accx[i] = 0.f;
      accy[i] = 0.f;
      accz[i] = 0.f;
    }
    for (int f = tid; f < ac.S * kNR; f += kHeavyThreads) grad[f] = g_row[ac.rcol[f >> 4] + (f & 15)];
    if (w == 0) build_block_table(H, ac, lane, bt_geo, bt_start);
    __syncthreads();
    // every block with triplets: its 32 dE/dG values (index 8a + z)
    for (int i = tid; i < np * 32; i += kHeavyThreads) {
      const int q = i >> 5, l = i & 31;
      if (bt_start[q + 1] > bt_start[q]) gf[q * 32 + l] = g_row[ac.acol[q] + l];
    }
    __syncthreads();
    float fi[3] = {0.f, 0.f, 0.f};
    float vir[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) vir[k] = 0.f;
    int sr = 0;
    for (int t = tid; t < nr; t += kHeavyThreads) {
      while (H.off_r[sr + 1] <= t) ++sr;
      const int j = lr[t];
      if (!NNP_IN_BOUNDS(ws.status, kSiteBwdNeighbour, j, ws.totals[0])) continue;
      radial_edge_bwd<VIR>(ws, ac, xi, d, j, ws.xyzq[j], grad + sr * kNR, inv_rc_r, fi, vir,
                           det ? ws.fr_det + (size_t)p * ws.cap_r + t : nullptr);
    }
    const int n_tri = bt_start[np];
    const int cp = w * n_lane + ((int)lane & (n_lane - 1));
    int bl = 0, cur = -1;
    int os = 0, cs = 0, ou = 0, cu = 0, same = 0;
    float inv_cs = 0.f, inv_cu = 0.f;
    auto triplet = [&](int t, float3& uj, float3& uk, int& aj, int& ak) -> bool {
      while (bt_start[bl + 1] <= t) ++bl;
      if (bl != cur) {
        cur = bl;
        const int4 g4 = bt_geo[bl];
        os = g4.x; cs = g4.y; ou = g4.z; cu = g4.w & 0xffff; same = (g4.w >> 16) & 1;
        inv_cs = rcp_approx((float)max(cs, 1));
        inv_cu = rcp_approx((float)max(cu, 1));   // decode corrects one step either way
      }
      int j, k;
      decode_pair_diag(t - bt_start[bl], same, cs, cu, inv_cs, inv_cu, &j, &k);
      const int tj = os + j, tk = ou + k;
      if (!NNP_IN_BOUNDS(ws.status, kSiteBwdTriplet, tj, na) ||
          !NNP_IN_BOUNDS(ws.status, kSiteBwdTriplet, tk, na))
        return false;
      triplet_bwd<ZETA>(ac, angv[tj], angv[tk], angf[tj], angf[tk], gall + bl * 8, uj, uk);
      aj = tj * n_acc + cp;
      ak = tk * n_acc + cp;
      return true;
    };
    if (!det) {
      for (int t = tid; t < n_tri; t += kHeavyThreads) {
        float3 uj, uk;
        int aj, ak;
        if (!triplet(t, uj, uk, aj, ak)) continue;
        atomicAdd(accx + aj, uj.x);
        atomicAdd(accy + aj, uj.y);
        atomicAdd(accz + aj, uj.z);
        atomicAdd(accx + ak, uk.x);
        atomicAdd(accy + ak, uk.y);
        atomicAdd(accz + ak, uk.z);
      }
    } else {
      // deterministic mode: within a warp the lanes add one after the other (the
      // warps add into their own copies)
      for (int t0 = w * 32; t0 < n_tri; t0 += kHeavyThreads) {
        float3 uj, uk;
        int aj = 0, ak = 0;
        const bool act = t0 + (int)lane < n_tri && triplet(t0 + (int)lane, uj, uk, aj, ak);
        for (int l = 0; l < 32; ++l) {
          if (act && (int)lane == l) {
            accx[aj] += uj.x; accy[aj] += uj.y; accz[aj] += uj.z;
            accx[ak] += uk.x; accy[ak] += uk.y; accz[ak] += uk.z;
          }
          __syncwarp();
        }
      }
    }
    __syncthreads();
    for (int t = tid; t < na; t += kHeavyThreads) {
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int c = 0; c < n_acc; ++c) {
        const int i = t * n_acc + c;
        a.x += accx[i];
        a.y += accy[i];
        a.z += accz[i];
      }
      const float4 v = angv[t];
      const int jt = __float_as_int(angf[t].w);
      if (det) ws.fa_det[(size_t)p * ws.cap_a + t] = make_float4(-a.x, -a.y, -a.z, 0.f);
      else if (NNP_IN_BOUNDS(ws.status, kSiteBwdNeighbour, jt, ws.totals[0]))
        atomicAdd(&ws.f_pos[jt], make_float4(-a.x, -a.y, -a.z, 0.f));
      fi[0] += a.x; fi[1] += a.y; fi[2] += a.z;
      if (VIR) {
        const float ux = v.x * v.w, uy = v.y * v.w, uz = v.z * v.w;
        vir[0] -= ux * a.x; vir[1] -= ux * a.y; vir[2] -= ux * a.z;
        vir[3] -= uy * a.x; vir[4] -= uy * a.y; vir[5] -= uy * a.z;
        vir[6] -= uz * a.x; vir[7] -= uz * a.y; vir[8] -= uz * a.z;
      }
    }
    // the centre's force and the virial: warp sums, then warp 0 over the warps
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      fi[0] += __shfl_xor_sync(kFull, fi[0], o);
      fi[1] += __shfl_xor_sync(kFull, fi[1], o);
      fi[2] += __shfl_xor_sync(kFull, fi[2], o);
#pragma unroll
      for (int k = 0; k < 9; ++k)
        if (VIR) vir[k] += __shfl_xor_sync(kFull, vir[k], o);
    }
    if (lane == 0) {
      red[w][0] = fi[0]; red[w][1] = fi[1]; red[w][2] = fi[2];
#pragma unroll
      for (int k = 0; k < 9; ++k) red[w][3 + k] = VIR ? vir[k] : 0.f;
    }
    __syncthreads();
    if (tid < 12) {
      float v = 0.f;
      for (int k = 0; k < kHeavyThreads / 32; ++k) v += red[k][tid];
      if (tid < 3) {
        if (det) reinterpret_cast<float*>(&ws.fs_det[p])[tid] = v;
        else atomicAdd(reinterpret_cast<float*>(&ws.f_pos[p]) + tid, v);
      } else if (VIR && d.in.virial) {
        if (det) ws.v_det[(size_t)p * 9 + (tid - 3)] = (double)v;
        else atomicAdd(d.in.virial + (tid - 3), (double)v);
      }
    }
  }
}

// ---------------------------------------------------------------- AEV -> first layer
// One CTA per 128-row tile of a species segment (BF16, one-network models):
// its 32 warps compute the AEV rows of the tile's atoms (four per warp, the
// same per-centre code as k_aev_fwd) straight into shared memory as BF16, in
// the 128-byte-swizzled K-major layout the tensor core reads, so the AEV never
// goes to HBM; then one thread streams the species' W1 by TMA in 64-wide K
// slices and issues tcgen05.mma (M = 128, N = h1) into tensor memory, and four
// warps apply the bias and CELU and write h1.  Rows past the segment's atom
// count are zero.
constexpr int kL1Warps = 32;
constexpr int kL1Blk = 128 * 128;          // one 64-column block of the A tile (bytes)
constexpr int kL1MaxSmem = 232448 - 16384;

struct AevL1Args {
  const float* b1;      // [S][h1]
  __nv_bfloat16* H1;    // [rows][h1]
  int h1;
  float alpha;
  int stage_bytes;      // one W1 slice: h1 x 64 BF16
};

__device__ __forceinline__ void put_tile(uint8_t* tile, int r, int f, float v) {
  const int blk = f >> 6, c = f & 63;
  uint8_t* row = tile + blk * kL1Blk + r * 128;
  const int off = ((((c >> 3) ^ (r & 7)) << 4) | ((c & 7) << 1));
  *reinterpret_cast<__nv_bfloat16*>(row + off) = __float2bfloat16_rn(v);
}

template <int ZETA>
__global__ void __launch_bounds__(kL1Warps * 32, 1)
k_aev_l1(const __grid_constant__ CUtensorMap tw1, Ws ws, AevConst ac, AevL1Args g) {
  using namespace tcu;
  extern __shared__ uint8_t smem_raw[];
  __shared__ ListHdr hdrs[kL1Warps];
  __shared__ __align__(8) uint64_t full_bar[2], empty_bar[2], done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  __shared__ uint8_t pair_su[kMaxSpecies * (kMaxSpecies + 1) / 2];
  const int w = threadIdx.x >> 5;
  const unsigned lane = threadIdx.x & 31;
  const int S = ac.S;
  const int row_tiles = ws.seg_start[S] / kTileM;
  if ((int)blockIdx.x >= row_tiles) return;    // uniform over the CTA
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nblk = ac.Dp / 64;
  uint8_t* tile = smem;
  uint8_t* ring = tile + nblk * kL1Blk;
  float4* stage = reinterpret_cast<float4*>(ring + 2 * g.stage_bytes) +
                  (size_t)w * aev_fwd_warp_f4(ws.cap_a, ws.cap_r);
  volatile int* abort_flag = &abort_sh;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&empty_bar[i], 1);
    }
    mbar_init(&done_bar, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)), "r"(256u) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fill_pair_table(pair_su, ac);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  const int m0 = blockIdx.x * kTileM;
  int sp = 0;
  while (sp + 1 < S && m0 >= ws.seg_start[sp + 1]) ++sp;
  const int seg_end = ws.seg_start[sp] + ws.species_count[sp];
  // ---- the tile's AEV rows into shared memory
  for (int r = w; r < kTileM; r += kL1Warps) {
    const int slot = m0 + r;
    if (slot < seg_end) {
      aev_centre<ZETA>(ws, ac, ws.slot_pos[slot], stage, hdrs[w], lane, pair_su,
                       [&](int f, float v) { put_tile(tile, r, f, v); });
    } else {
      for (int f = (int)lane; f < ac.Dp; f += 32) put_tile(tile, r, f, 0.f);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor core
  __syncthreads();
  // ---- first layer: W1 of species sp by TMA, MMAs by one thread
  if (w == 0 && lane == 0) {
    const int nk = nblk;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(g.h1 >> 3) << 17) |
                           ((uint32_t)(kTileM >> 4) << 24);
    bool ok = true;
    int issued = 0;
    for (; issued < 2 && issued < nk; ++issued) {
      mbar_expect_tx(&full_bar[issued], (unsigned)g.stage_bytes);
      tma_load_3d(ring + issued * g.stage_bytes, &tw1, &full_bar[issued], issued * 64, 0, sp);
    }
    for (int kb = 0; kb < nk && ok; ++kb) {
      const int st = kb & 1;
      if (!mbar_wait(&full_bar[st], (kb >> 1) & 1, abort_flag)) { ok = false; break; }
      tc_fence_after();
      const uint64_t ad = sw128_desc(smem_u32(tile + kb * kL1Blk));
      const uint64_t bd = sw128_desc(smem_u32(ring + st * g.stage_bytes));
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        umma_bf16(tmem, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc, (kb > 0 || kk > 0) ? 1u : 0u);
      umma_commit(&empty_bar[st]);
      if (issued < nk) {
        if (!mbar_wait(&empty_bar[st], (kb >> 1) & 1, abort_flag)) { ok = false; break; }
        mbar_expect_tx(&full_bar[st], (unsigned)g.stage_bytes);
        tma_load_3d(ring + st * g.stage_bytes, &tw1, &full_bar[st], issued * 64, 0, sp);
        ++issued;
      }
    }
    umma_commit(&done_bar);   // arrives when every MMA issued above has completed
    if (!ok) {
      // every issued copy lands before the CTA may exit
      for (int k = issued - 2 < 0 ? 0 : issued - 2; k < issued; ++k)
        mbar_drain(&full_bar[k & 1], (k >> 1) & 1);
    }
  }
  // ---- epilogue: bias, CELU, h1 (TMEM lanes 32 w .. of warps 0-3)
  if (w < 4) {
    if (mbar_wait(&done_bar, 0, abort_flag)) {
      tc_fence_after();
      const int r = w * 32 + (int)lane;
      const uint32_t trow = tmem + ((uint32_t)(w * 32) << 16);
      const float* bias = g.b1 + (size_t)sp * g.h1;
      const float alpha = g.alpha, inv_alpha = 1.f / g.alpha;
      for (int c0 = 0; c0 < g.h1; c0 += 16) {
        float v[16];
        tmem_ld16(trow + (uint32_t)c0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float z = v[i] + __ldg(bias + c0 + i);
          v[i] = z > 0.f ? z : alpha * (__expf(z * inv_alpha) - 1.f);
        }
        store_bf16x16(g.H1 + (size_t)(m0 + r) * g.h1 + c0, v);
      }
    } else {
      mbar_drain(&done_bar, 0);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicOr(ws.status, kStTimeout);
  if (w == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u) : "memory");
}

size_t aev_l1_smem(const Ws& ws, const AevConst& ac, int h1) {
  return (size_t)(ac.Dp / 64) * kL1Blk + 2 * (size_t)h1 * 64 * 2 +
         (size_t)kL1Warps * aev_fwd_warp_f4(ws.cap_a, ws.cap_r) * sizeof(float4) + 1024;
}

}  // namespace

size_t aev_fwd_smem(const Ws& ws) {
  return (size_t)kWarps * aev_fwd_warp_f4(ws.cap_a, ws.cap_r) * sizeof(float4);
}
// angular neighbours the warp-per-centre backward handles; centres with more go
// to the CTA-per-centre kernel
constexpr int kLightCapA = 48;
static int light_cap(const Ws& ws) { return std::min(ws.cap_a, kLightCapA); }

size_t aev_bwd_smem(const Ws& ws, int n_pairs) {
  const int cap_l = light_cap(ws);
  return (size_t)kWarps * aev_bwd_warp_f4(cap_l, n_pairs, aev_bwd_copies(cap_l, n_pairs)) *
         sizeof(float4);
}

// lane copies per warp of the CTA-per-centre kernel's accumulators: as many as
// keep its shared memory within 96 KiB (two CTAs per SM), at most 4
static int heavy_log_n(const Ws& ws, int n_pairs) {
  for (int l = 2; l > 0; --l)
    if (aev_bwd_heavy_smem(ws.cap_a, n_pairs, 1 << l) <= 96 * 1024) return l;
  return 0;
}
static size_t heavy_smem(const Ws& ws, int n_pairs) {
  return aev_bwd_heavy_smem(ws.cap_a, n_pairs, 1 << heavy_log_n(ws, n_pairs));
}

// grid of the persistent warp-per-centre kernels: four CTAs per SM at most,
// fewer for small batches
static int centre_grid(int n_in) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
  }
  return std::max(1, std::min((n_in + kWarps - 1) / kWarps, 4 * sms));
}

void launch_aev_fwd(const Ws& ws, int n_in, const AevConst& ac, cudaStream_t st) {
  if (n_in <= 0) return;
  const size_t sm = aev_fwd_smem(ws);
  const int grid = centre_grid(n_in);
  if (ac.zeta == 32) k_aev_fwd<32><<<grid, kWarps * 32, sm, st>>>(ws, ac);
  else k_aev_fwd<0><<<grid, kWarps * 32, sm, st>>>(ws, ac);
}

void launch_aev_fill(const Ws& ws, const AevConst& ac, cudaStream_t st) {
  if (!ws.row_mask) return;
  k_aev_fill<<<(ws.row_cap + 7) / 8, 256, 0, st>>>(ws, ac);
}

void launch_aev_bwd(const Ws& ws, int n_in, const AevConst& ac, int want_virial,
                    cudaStream_t st) {
  if (n_in <= 0) return;
  const int cap_l = light_cap(ws);
  const size_t sm = aev_bwd_smem(ws, ac.n_pairs);
  const int copies = aev_bwd_copies(cap_l, ac.n_pairs);
  const int log_r = copies == 4 ? 2 : copies == 2 ? 1 : 0;
  const int grid = centre_grid(n_in);
  if (ac.zeta == 32) {
    if (want_virial) k_aev_bwd<32, true><<<grid, kWarps * 32, sm, st>>>(ws, ac, log_r, cap_l);
    else k_aev_bwd<32, false><<<grid, kWarps * 32, sm, st>>>(ws, ac, log_r, cap_l);
  } else {
    if (want_virial) k_aev_bwd<0, true><<<grid, kWarps * 32, sm, st>>>(ws, ac, log_r, cap_l);
    else k_aev_bwd<0, false><<<grid, kWarps * 32, sm, st>>>(ws, ac, log_r, cap_l);
  }
  // no centre can have more neighbours or live species-pair blocks than the warps take
  if (ws.cap_a <= cap_l && ac.n_pairs <= kGallBlocks) return;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int hgrid = std::max(1, std::min(n_in, 4 * std::max(sms, 1)));
  const size_t hs = heavy_smem(ws, ac.n_pairs);
  const int log_n = heavy_log_n(ws, ac.n_pairs);
  if (ac.zeta == 32) {
    if (want_virial) k_aev_bwd_heavy<32, true><<<hgrid, kHeavyThreads, hs, st>>>(ws, ac, log_n);
    else k_aev_bwd_heavy<32, false><<<hgrid, kHeavyThreads, hs, st>>>(ws, ac, log_n);
  } else {
    if (want_virial) k_aev_bwd_heavy<0, true><<<hgrid, kHeavyThreads, hs, st>>>(ws, ac, log_n);
    else k_aev_bwd_heavy<0, false><<<hgrid, kHeavyThreads, hs, st>>>(ws, ac, log_n);
  }
}

// raise (never lower) the dynamic shared-memory limit of the AEV kernels to what
// a launch over `ws` needs
cudaError_t aev_ensure_smem(const Ws& ws) {
  // the backward kernel's size depends on the species-pair count through the
  // number of accumulator copies: take the largest over every model size
  int need_b = 0;
  for (int np = 1; np <= kMaxSpecies * (kMaxSpecies + 1) / 2; ++np)
    need_b = std::max(need_b, (int)aev_bwd_smem(ws, np));
  const int need_f = (int)aev_fwd_smem(ws);
  int need_h = 0;
  for (int np = 1; np <= kMaxSpecies * (kMaxSpecies + 1) / 2; ++np)
    need_h = std::max(need_h, (int)heavy_smem(ws, np));
  const void* fwd[2] = {(const void*)k_aev_fwd<32>, (const void*)k_aev_fwd<0>};
  const void* bwd[4] = {(const void*)k_aev_bwd<32, false>, (const void*)k_aev_bwd<32, true>,
                        (const void*)k_aev_bwd<0, false>, (const void*)k_aev_bwd<0, true>};
  const void* hvy[4] = {(const void*)k_aev_bwd_heavy<32, false>,
                        (const void*)k_aev_bwd_heavy<32, true>,
                        (const void*)k_aev_bwd_heavy<0, false>,
                        (const void*)k_aev_bwd_heavy<0, true>};
  for (int pass = 0; pass < 3; ++pass)
    for (int i = 0; i < (pass == 0 ? 2 : 4); ++i) {
      const void* fn = pass == 0 ? fwd[i] : pass == 1 ? bwd[i] : hvy[i];
      const int need = pass == 0 ? need_f : pass == 1 ? need_b : need_h;
      cudaFuncAttributes attr;
      cudaError_t e = cudaFuncGetAttributes(&attr, fn);
      if (e != cudaSuccess) return e;
      if (attr.maxDynamicSharedSizeBytes < need) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
        if (e != cudaSuccess) return e;
      }
    }
  return cudaSuccess;
}


bool aev_l1_supported(const Ws& ws, const AevConst& ac, int E, int h1) {
  return E == 1 && ac.Dp % 64 == 0 && h1 % 16 == 0 && h1 >= 16 && h1 <= 256 && ws.slot_pos &&
         aev_l1_smem(ws, ac, h1) <= (size_t)kL1MaxSmem;
}

void launch_aev_l1(const Ws& ws, const AevConst& ac, const void* w1_bf16, const float* b1,
                   void* H1, int h1, float alpha, cudaStream_t st) {
  // W1 of every species [S][h1][Dp] BF16: dims (Dp, h1, S), box (64, h1, 1)
  CUtensorMap m;
  if (!tcu::make_map(&m, w1_bf16, ac.Dp, h1, ac.S, ac.Dp, (uint64_t)ac.Dp * h1, (uint32_t)h1, 1)) return;
  AevL1Args g{};
  g.b1 = b1;
  g.H1 = static_cast<__nv_bfloat16*>(H1);
  g.h1 = h1;
  g.alpha = alpha;
  g.stage_bytes = h1 * 64 * 2;
  const size_t sm = aev_l1_smem(ws, ac, h1);
  const int grid = (ws.row_cap + tcu::kTileM - 1) / tcu::kTileM;
  if (ac.zeta == 32) k_aev_l1<32><<<grid, kL1Warps * 32, sm, st>>>(m, ws, ac, g);
  else k_aev_l1<0><<<grid, kL1Warps * 32, sm, st>>>(m, ws, ac, g);
}

cudaError_t aev_l1_ensure_smem(const Ws& ws, const AevConst& ac, int h1) {
  const int need = (int)std::min(aev_l1_smem(ws, ac, h1), (size_t)kL1MaxSmem);
  for (const void* fn : {(const void*)k_aev_l1<32>, (const void*)k_aev_l1<0>}) {
    cudaFuncAttributes attr;
    cudaError_t e = cudaFuncGetAttributes(&attr, fn);
    if (e != cudaSuccess) return e;
    if (attr.maxDynamicSharedSizeBytes < need) {
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace nnp
