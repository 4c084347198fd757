// Atomic environment vectors (paper Eqs. 3-5) and their backward to forces.
//
// One warp per centre atom.  The neighbour geometry of the centre is computed
// once per neighbour (lane-parallel) and staged in shared memory; then
//   radial  (Eq. 4): two half-warps take alternate neighbours of one species, a
//           lane owns one Gaussian shell r; a final xor-16 shuffle sums the two
//           halves and lanes 0..15 write the 16 features of the block.
//   angular (Eq. 5): the warp is four groups of eight lanes; a group takes every
//           fourth (j, k) pair of one unordered species pair, lane z of the group
//           owns the angle section theta_z and the four distance shells a; the
//           four groups are summed with xor-8/16 shuffles and lane (a, z) writes
//           feature 8a + z, so each 32-feature block is one coalesced 128-byte
//           store.
// The angular factor uses cos(theta - theta_z) = cos theta cos theta_z +
// sin theta sin theta_z with sin theta from the cross product (no acos), and
// (1 + cos(theta - theta_z))^zeta by repeated squaring (integer zeta).
//
// Backward (forces F = -dE/dr): radial edges are done lane-per-neighbour; every
// angular (j, k) pair is reduced over its group to dE/dcos, dE/dRbar and
// dE/d(f_j f_k), turned into dE/du_j and dE/du_k and added to per-neighbour
// accumulators in shared memory; each neighbour then receives one vector atomic.
#include "nnp_internal.cuh"

namespace nnp {

namespace {

constexpr int kWarps = 8;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kPi = 3.14159265358979f;

__device__ __forceinline__ float fast_exp2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float ipow(float x, int e) {
  float r = 1.f;
  while (e) {
    if (e & 1) r *= x;
    x *= x;
    e >>= 1;
  }
  return r;
}

struct Geo {
  float dx, dy, dz, r;
};

__device__ __forceinline__ Geo pair_geo(const float4& xi, const float4& xj, const SysDev& d) {
  float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
  if (d.in.periodic) {
    float n;
    n = rintf(dx * (1.f / d.in.box_hi[0])); dx = fmaf(-n, d.in.box_hi[0], dx); dx = fmaf(-n, d.in.box_lo[0], dx);
    n = rintf(dy * (1.f / d.in.box_hi[1])); dy = fmaf(-n, d.in.box_hi[1], dy); dy = fmaf(-n, d.in.box_lo[1], dy);
    n = rintf(dz * (1.f / d.in.box_hi[2])); dz = fmaf(-n, d.in.box_hi[2], dz); dz = fmaf(-n, d.in.box_lo[2], dz);
  }
  Geo g;
  g.dx = dx; g.dy = dy; g.dz = dz;
  g.r = sqrtf(dx * dx + dy * dy + dz * dz);
  return g;
}

// cosine cutoff (Eq. 3) and its derivative
__device__ __forceinline__ float fcut(float r, float rc) {
  return r < rc ? 0.5f * cospif(r / rc) + 0.5f : 0.f;
}
__device__ __forceinline__ float fcut_d(float r, float rc) {
  return r < rc ? -0.5f * (kPi / rc) * sinpif(r / rc) : 0.f;
}

// species offsets of a centre's lists from its header
__device__ __forceinline__ void list_offsets(const uint16_t* hdr, int S, unsigned lane,
                                             int* off_r, int* cnt_r, int* off_a, int* cnt_a) {
  int cr = (lane < (unsigned)S) ? hdr[lane] : 0;
  int ca = (lane < (unsigned)S) ? hdr[8 + lane] : 0;
  int ir = cr, ia = ca;
  for (int o = 1; o < 8; o <<= 1) {
    int u = __shfl_up_sync(0xffffffffu, ir, o);
    int v = __shfl_up_sync(0xffffffffu, ia, o);
    if ((int)lane >= o) { ir += u; ia += v; }
  }
#pragma unroll
  for (int s = 0; s < kMaxSpecies; ++s) {
    cnt_r[s] = __shfl_sync(0xffffffffu, cr, s);
    cnt_a[s] = __shfl_sync(0xffffffffu, ca, s);
    off_r[s] = __shfl_sync(0xffffffffu, ir - cr, s);
    off_a[s] = __shfl_sync(0xffffffffu, ia - ca, s);
  }
}

// iterate the (j, k) pairs of one species-pair block for group g of 4:
// same species: j < k in [0, c); different species: j in [0, cs), k in [0, ct)
struct PairIter {
  int j, k, cs, ct, same;
  __device__ __forceinline__ void start(int g, int cs_, int ct_, int same_) {
    cs = cs_; ct = ct_; same = same_;
    if (same) {
      j = 0; k = 1 + g;
      while (j < cs && k >= cs) { ++j; k = k - cs + j + 1; }
    } else {
      j = ct > 0 ? g / ct : cs;
      k = ct > 0 ? g % ct : 0;
    }
  }
  __device__ __forceinline__ bool valid() const { return same ? (j < cs - 1 && k < cs) : (j < cs); }
  __device__ __forceinline__ void next() {
    k += 4;
    if (same) {
      while (j < cs && k >= cs) { ++j; k = k - cs + j + 1; }
    } else {
      while (k >= ct && j < cs) { k -= ct; ++j; }
    }
  }
};

// sin(theta) with theta = acos(k cos_hat): sqrt(1 - k^2 cos_hat^2) written as
// sqrt(|u_j x u_k|^2 + (1 - k^2) cos_hat^2), which keeps full relative accuracy
// for nearly collinear triplets (where 1 - cos^2 cancels)
__device__ __forceinline__ float sin_theta(const float4& a, const float4& b, float chat, float k) {
  const float cx = a.y * b.z - a.z * b.y;
  const float cy = a.z * b.x - a.x * b.z;
  const float cz = a.x * b.y - a.y * b.x;
  const float s2 = cx * cx + cy * cy + cz * cz;
  return sqrtf(fmaf(1.f - k * k, chat * chat, s2));
}

__device__ __forceinline__ float pick4(const float v[4], int i) {
  float r = v[0];
  r = (i == 1) ? v[1] : r;
  r = (i == 2) ? v[2] : r;
  r = (i == 3) ? v[3] : r;
  return r;
}

__global__ void __launch_bounds__(kWarps * 32)
k_aev_fwd(Ws ws, AevConst ac) {
  extern __shared__ float4 sm4[];
  const int w = threadIdx.x >> 5;
  const unsigned lane = threadIdx.x & 31;
  const int p = blockIdx.x * kWarps + w;
  if (p >= ws.totals[0]) return;
  // per-warp staging: angular (u, R) and fc, radial (R, fc)
  float4* angv = sm4 + (size_t)w * (ws.cap_a + ws.cap_a / 4 + ws.cap_r / 2 + 2);
  float* angf = reinterpret_cast<float*>(angv + ws.cap_a);
  float2* rad = reinterpret_cast<float2*>(angf + ws.cap_a + 4);

  const float4 xi = ws.xyzq[p];
  const SysDev& d = ws.sys[ws.pos_sys[p]];
  const int slot = ws.pos_slot[p];
  float* G = ws.aev + (size_t)slot * ac.Dp;
  int off_r[kMaxSpecies], cnt_r[kMaxSpecies], off_a[kMaxSpecies], cnt_a[kMaxSpecies];
  list_offsets(ws.nb_cnt + (size_t)p * 16, ac.S, lane, off_r, cnt_r, off_a, cnt_a);
  const int nr_tot = off_r[ac.S - 1] + cnt_r[ac.S - 1];
  const int na_tot = off_a[ac.S - 1] + cnt_a[ac.S - 1];
  const int* lr = ws.nb_r + (size_t)p * ws.cap_r;
  const int* la = ws.nb_a + (size_t)p * ws.cap_a;
  for (int t = lane; t < nr_tot; t += 32) {
    const Geo g = pair_geo(xi, ws.xyzq[lr[t]], d);
    rad[t] = make_float2(g.r, fcut(g.r, ac.rc_r));
  }
  for (int t = lane; t < na_tot; t += 32) {
    const Geo g = pair_geo(xi, ws.xyzq[la[t]], d);
    const float inv = 1.f / g.r;
    angv[t] = make_float4(g.dx * inv, g.dy * inv, g.dz * inv, g.r);
    angf[t] = fcut(g.r, ac.rc_a);
  }
  __syncwarp();
  // ---- radial, Eq. 4
  const float cr_ = -ac.eta_r * kLog2e;
  const float my_shf = ac.shf_r[lane & 15];
  const int half = lane >> 4;
  for (int s = 0; s < ac.S; ++s) {
    float acc = 0.f;
    const float2* rs = rad + off_r[s];
    for (int t = half; t < cnt_r[s]; t += 2) {
      const float2 q = rs[t];
      const float x = q.x - my_shf;
      acc = fmaf(fast_exp2(cr_ * x * x), q.y, acc);
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 16);
    if (lane < 16) G[s * kNR + lane] = acc;
  }
  // ---- angular, Eq. 5
  const int grp = lane >> 3, z = lane & 7;
  const float cz = ac.cos_z[z], sz = ac.sin_z[z];
  const float ca_ = -ac.eta_a * kLog2e;
  const float sa0 = ac.shf_a[0], sa1 = ac.shf_a[1], sa2 = ac.shf_a[2], sa3 = ac.shf_a[3];
  int pidx = 0;
  for (int s = 0; s < ac.S; ++s)
    for (int u = s; u < ac.S; ++u, ++pidx) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      PairIter it;
      it.start(grp, cnt_a[s], cnt_a[u], s == u);
      const int os = off_a[s], ou = off_a[u];
      for (; it.valid(); it.next()) {
        const float4 vj = angv[os + it.j];
        const float4 vk = angv[ou + it.k];
        const float fjk = angf[os + it.j] * angf[ou + it.k];
        const float chat = vj.x * vk.x + vj.y * vk.y + vj.z * vk.z;
        const float c = ac.cos_scale * chat;
        const float sn = sin_theta(vj, vk, chat, ac.cos_scale);
        const float base = 1.f + c * cz + sn * sz;
        const float f = ac.ang_pre * ipow(base, ac.zeta) * fjk;
        const float rb = 0.5f * (vj.w + vk.w);
        float x;
        x = rb - sa0; acc[0] = fmaf(fast_exp2(ca_ * x * x), f, acc[0]);
        x = rb - sa1; acc[1] = fmaf(fast_exp2(ca_ * x * x), f, acc[1]);
        x = rb - sa2; acc[2] = fmaf(fast_exp2(ca_ * x * x), f, acc[2]);
        x = rb - sa3; acc[3] = fmaf(fast_exp2(ca_ * x * x), f, acc[3]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], 8);
        acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], 16);
      }
      G[ac.S * kNR + pidx * 32 + lane] = pick4(acc, grp);
    }
  for (int f = ac.D + lane; f < ac.Dp; f += 32) G[f] = 0.f;
}

__global__ void __launch_bounds__(kWarps * 32)
k_aev_bwd(Ws ws, AevConst ac, int want_virial) {
  extern __shared__ float4 sm4[];
  const int w = threadIdx.x >> 5;
  const unsigned lane = threadIdx.x & 31;
  const int p = blockIdx.x * kWarps + w;
  if (p >= ws.totals[0]) return;
  // per-warp staging: angular (u, R), (fc, dfc), accumulators; radial dE/dG
  float4* angv = sm4 + (size_t)w * (3 * ws.cap_a + 32);
  float4* angf = angv + ws.cap_a;          // fc, dfc
  float4* acc3 = angf + ws.cap_a;          // dE/du per angular neighbour
  float* grad = reinterpret_cast<float*>(acc3 + ws.cap_a);  // S*16 radial dE/dG

  const float4 xi = ws.xyzq[p];
  const int b = ws.pos_sys[p];
  const SysDev& d = ws.sys[b];
  const int slot = ws.pos_slot[p];
  const float* g_row = ws.dEdG + (size_t)slot * ac.Dp;
  int off_r[kMaxSpecies], cnt_r[kMaxSpecies], off_a[kMaxSpecies], cnt_a[kMaxSpecies];
  list_offsets(ws.nb_cnt + (size_t)p * 16, ac.S, lane, off_r, cnt_r, off_a, cnt_a);
  const int nr_tot = off_r[ac.S - 1] + cnt_r[ac.S - 1];
  const int na_tot = off_a[ac.S - 1] + cnt_a[ac.S - 1];
  const int* lr = ws.nb_r + (size_t)p * ws.cap_r;
  const int* la = ws.nb_a + (size_t)p * ws.cap_a;
  for (int f = lane; f < ac.S * kNR; f += 32) grad[f] = g_row[f];
  for (int t = lane; t < na_tot; t += 32) {
    const Geo g = pair_geo(xi, ws.xyzq[la[t]], d);
    const float inv = 1.f / g.r;
    angv[t] = make_float4(g.dx * inv, g.dy * inv, g.dz * inv, g.r);
    angf[t] = make_float4(fcut(g.r, ac.rc_a), fcut_d(g.r, ac.rc_a), 0.f, 0.f);
    acc3[t] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncwarp();
  float fi[3] = {0.f, 0.f, 0.f};
  float vir[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) vir[k] = 0.f;
  // ---- radial edges, one lane per neighbour
  const float cr_ = -ac.eta_r * kLog2e;
  {
    int s = 0;
    for (int t = lane; t < nr_tot; t += 32) {
      while (s + 1 < ac.S && t >= off_r[s + 1]) ++s;
      const int j = lr[t];
      const Geo g = pair_geo(xi, ws.xyzq[j], d);
      const float fc = fcut(g.r, ac.rc_r), dfc = fcut_d(g.r, ac.rc_r);
      float dEdR = 0.f;
      const float* gs = grad + s * kNR;
#pragma unroll
      for (int r = 0; r < kNR; ++r) {
        const float x = g.r - ac.shf_r[r];
        const float e = fast_exp2(cr_ * x * x);
        dEdR = fmaf(gs[r], e * fmaf(-2.f * ac.eta_r * x, fc, dfc), dEdR);
      }
      const float sc = dEdR / g.r;
      const float gx = sc * g.dx, gy = sc * g.dy, gz = sc * g.dz;
      atomicAdd(&ws.f_pos[j], make_float4(-gx, -gy, -gz, 0.f));
      fi[0] += gx; fi[1] += gy; fi[2] += gz;
      if (want_virial) {
        vir[0] -= g.dx * gx; vir[1] -= g.dx * gy; vir[2] -= g.dx * gz;
        vir[3] -= g.dy * gx; vir[4] -= g.dy * gy; vir[5] -= g.dy * gz;
        vir[6] -= g.dz * gx; vir[7] -= g.dz * gy; vir[8] -= g.dz * gz;
      }
    }
  }
  // ---- angular (j, k) pairs
  const int grp = lane >> 3, z = lane & 7;
  const float cz = ac.cos_z[z], sz = ac.sin_z[z];
  const float ca_ = -ac.eta_a * kLog2e;
  const float two_eta_a = 2.f * ac.eta_a;
  const float sa[4] = {ac.shf_a[0], ac.shf_a[1], ac.shf_a[2], ac.shf_a[3]};
  int pidx = 0;
  for (int s = 0; s < ac.S; ++s)
    for (int u = s; u < ac.S; ++u, ++pidx) {
      if (cnt_a[s] == 0 || cnt_a[u] == 0 || (s == u && cnt_a[s] < 2)) continue;
      const float* gb = g_row + ac.S * kNR + pidx * 32;
      const float G0 = gb[0 * 8 + z], G1 = gb[1 * 8 + z], G2 = gb[2 * 8 + z], G3 = gb[3 * 8 + z];
      PairIter it;
      it.start(grp, cnt_a[s], cnt_a[u], s == u);
      const int os = off_a[s], ou = off_a[u];
      // all lanes of a group iterate together; groups may differ in trip count
      for (; it.valid(); it.next()) {
        const int tj = os + it.j, tk = ou + it.k;
        const float4 vj = angv[tj], vk = angv[tk];
        const float4 fj4 = angf[tj], fk4 = angf[tk];
        const float chat = vj.x * vk.x + vj.y * vk.y + vj.z * vk.z;
        const float c = ac.cos_scale * chat;
        const float sn = fmaxf(sin_theta(vj, vk, chat, ac.cos_scale), 1e-6f);
        const float base = 1.f + c * cz + sn * sz;
        const float B1 = ipow(base, ac.zeta - 1);
        const float B = B1 * base;
        const float dBdc = (float)ac.zeta * B1 * (cz - sz * c / sn);
        const float rb = 0.5f * (vj.w + vk.w);
        float P = 0.f, Q = 0.f, x, e;
        x = rb - sa[0]; e = fast_exp2(ca_ * x * x); P = fmaf(G0, e, P); Q = fmaf(G0, -two_eta_a * x * e, Q);
        x = rb - sa[1]; e = fast_exp2(ca_ * x * x); P = fmaf(G1, e, P); Q = fmaf(G1, -two_eta_a * x * e, Q);
        x = rb - sa[2]; e = fast_exp2(ca_ * x * x); P = fmaf(G2, e, P); Q = fmaf(G2, -two_eta_a * x * e, Q);
        x = rb - sa[3]; e = fast_exp2(ca_ * x * x); P = fmaf(G3, e, P); Q = fmaf(G3, -two_eta_a * x * e, Q);
        const float fjk = fj4.x * fk4.x;
        float tc = ac.ang_pre * dBdc * P * fjk;   // dE/dc (c = cos_scale * chat)
        float tR = ac.ang_pre * B * Q * fjk;      // dE/dRbar
        float tf = ac.ang_pre * B * P;            // dE/d(fj fk)
        const unsigned gmask = 0xffu << (grp * 8);
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
          tc += __shfl_xor_sync(gmask, tc, o);
          tR += __shfl_xor_sync(gmask, tR, o);
          tf += __shfl_xor_sync(gmask, tf, o);
        }
        if (z < 2) {
          const float dEdchat = ac.cos_scale * tc;
          const float4 va = (z == 0) ? vj : vk;   // this lane's edge
          const float4 vb = (z == 0) ? vk : vj;
          const float radial = 0.5f * tR + tf * ((z == 0) ? fj4.y * fk4.x : fj4.x * fk4.y);
          const float sc = dEdchat / va.w;
          const float gx = sc * (vb.x - chat * va.x) + radial * va.x;
          const float gy = sc * (vb.y - chat * va.y) + radial * va.y;
          const float gz = sc * (vb.z - chat * va.z) + radial * va.z;
          float4* A = acc3 + ((z == 0) ? tj : tk);
          atomicAdd(&A->x, gx);
          atomicAdd(&A->y, gy);
          atomicAdd(&A->z, gz);
        }
      }
    }
  __syncwarp();
  for (int t = lane; t < na_tot; t += 32) {
    const float4 a = acc3[t];
    const float4 v = angv[t];
    atomicAdd(&ws.f_pos[la[t]], make_float4(-a.x, -a.y, -a.z, 0.f));
    fi[0] += a.x; fi[1] += a.y; fi[2] += a.z;
    if (want_virial) {
      const float ux = v.x * v.w, uy = v.y * v.w, uz = v.z * v.w;
      vir[0] -= ux * a.x; vir[1] -= ux * a.y; vir[2] -= ux * a.z;
      vir[3] -= uy * a.x; vir[4] -= uy * a.y; vir[5] -= uy * a.z;
      vir[6] -= uz * a.x; vir[7] -= uz * a.y; vir[8] -= uz * a.z;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fi[0] += __shfl_xor_sync(0xffffffffu, fi[0], o);
    fi[1] += __shfl_xor_sync(0xffffffffu, fi[1], o);
    fi[2] += __shfl_xor_sync(0xffffffffu, fi[2], o);
  }
  if (lane == 0) atomicAdd(&ws.f_pos[p], make_float4(fi[0], fi[1], fi[2], 0.f));
  if (want_virial && d.in.virial) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      float v = vir[k];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) atomicAdd(d.in.virial + k, (double)v);
    }
  }
}

}  // namespace

size_t aev_fwd_smem(const Ws& ws) {
  return (size_t)kWarps * (ws.cap_a + ws.cap_a / 4 + ws.cap_r / 2 + 2) * sizeof(float4);
}
size_t aev_bwd_smem(const Ws& ws) {
  return (size_t)kWarps * (3 * ws.cap_a + 32) * sizeof(float4);
}

void launch_aev_fwd(const Ws& ws, int n_in, const AevConst& ac, cudaStream_t st) {
  if (n_in <= 0) return;
  const size_t sm = aev_fwd_smem(ws);
  k_aev_fwd<<<(n_in + kWarps - 1) / kWarps, kWarps * 32, sm, st>>>(ws, ac);
}

void launch_aev_bwd(const Ws& ws, int n_in, const AevConst& ac, int want_virial,
                    cudaStream_t st) {
  if (n_in <= 0) return;
  const size_t sm = aev_bwd_smem(ws);
  k_aev_bwd<<<(n_in + kWarps - 1) / kWarps, kWarps * 32, sm, st>>>(ws, ac, want_virial);
}

cudaError_t aev_set_smem_limits(const Ws& ws) {
  cudaError_t e = cudaFuncSetAttribute(k_aev_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)aev_fwd_smem(ws));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_aev_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)aev_bwd_smem(ws));
}

}  // namespace nnp
