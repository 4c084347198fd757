// Double backward of the potential: the vector-Jacobian product of the forces,
// for training by force matching (loss L(E, F), v = dL/dF, gE = dL/dE).
//
//   dL/dr      = -gE F + d/de F(r + e v)            (a Hessian-vector product)
//   dL/dtheta  = gE dE/dtheta - d/dtheta [ sum_i dE_i/dG_i . u_i ],  u_i = J_i v
//
// Kernels (FP32):
//   k_gather_v       v in packed (cell) order
//   k_aev_jvp        u_i = d/de G_i(r + e v): the forward AEV differentiated along
//                    v (same lane-per-triplet layout as the forward)
//   k_vjp_out3 /
//   k_vjp_delta      element-wise steps of the network's forward-over-reverse
//                    pass (primal deltas and their tangents)
//   k_aev_bwd_dual   the AEV backward in dual-number arithmetic: primal inputs
//                    (r, dE/dG) with tangents (v, q = H_e u); its tangent output is
//                    d/de F
//   k_wgrad          per-species weight and bias gradients summed over rows
//   k_vjp_scatter    dL/dr back to the caller's atom order
#include <algorithm>

#include "mlp.cuh"
#include "nnp_internal.cuh"
#include "vjp.cuh"

namespace nnp {

namespace {

constexpr int kWarps = 8;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kPi = 3.14159265358979f;
constexpr unsigned kFull = 0xffffffffu;

// forward-mode dual number (value, tangent)
struct Df {
  float v, d;
};
__device__ __forceinline__ Df dd(float v, float d = 0.f) { return Df{v, d}; }
__device__ __forceinline__ Df operator+(Df a, Df b) { return Df{a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Df operator-(Df a, Df b) { return Df{a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Df operator*(Df a, Df b) { return Df{a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Df operator*(float s, Df a) { return Df{s * a.v, s * a.d}; }
__device__ __forceinline__ Df operator/(Df a, Df b) {
  const float inv = 1.f / b.v;
  return Df{a.v * inv, (a.d - a.v * inv * b.d) * inv};
}
__device__ __forceinline__ Df dsqrt(Df a) {
  const float s = sqrtf(a.v);
  return Df{s, a.d * 0.5f / s};
}
__device__ __forceinline__ float fast_exp2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ Df dexp2(Df a) {
  const float e = fast_exp2(a.v);
  return Df{e, e * kLn2 * a.d};
}

__device__ __forceinline__ float ipowf(float x, int e) {
  float r = 1.f;
  while (e) {
    if (e & 1) r *= x;
    x *= x;
    e >>= 1;
  }
  return r;
}

struct Geo {
  float dx, dy, dz;
};

__device__ __forceinline__ Geo disp(const float4& xi, const float4& xj, const SysDev& d) {
  float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
  if (d.in.periodic) {
    float n;
    n = rintf(dx * d.in.inv_box[0]); dx = fmaf(-n, d.in.box_hi[0], dx); dx = fmaf(-n, d.in.box_lo[0], dx);
    n = rintf(dy * d.in.inv_box[1]); dy = fmaf(-n, d.in.box_hi[1], dy); dy = fmaf(-n, d.in.box_lo[1], dy);
    n = rintf(dz * d.in.inv_box[2]); dz = fmaf(-n, d.in.box_hi[2], dz); dz = fmaf(-n, d.in.box_lo[2], dz);
  }
  return Geo{dx, dy, dz};
}

// cosine cutoff (Eq. 3) and its first two derivatives
__device__ __forceinline__ void fcut3(float r, float rc, float* f, float* df, float* ddf) {
  if (r < rc) {
    const float a = r / rc;
    *f = 0.5f * cospif(a) + 0.5f;
    *df = -0.5f * (kPi / rc) * sinpif(a);
    *ddf = -0.5f * (kPi / rc) * (kPi / rc) * cospif(a);
  } else {
    *f = *df = *ddf = 0.f;
  }
}

struct ListHdr {
  int off_r[kMaxSpecies + 1], off_a[kMaxSpecies + 1];
};

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

__device__ __forceinline__ void decode_pair(int t, int same, int c, int cu, float inv_cu, int* j, int* k) {
  if (same) {
    const float b = 2.f * c - 1.f;
    int jj = (int)((b - sqrtf(fmaxf(b * b - 8.f * t, 0.f))) * 0.5f);
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

__global__ void k_gather_v(Ws ws, VjpBufs vb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ws.totals[0]) return;
  const int b = ws.pos_sys[p];
  const int local = ws.pos_src[p] - ws.sys[b].in.in_base;
  const float* v = ws.sys[b].in.dLdF;
  vb.v_pos[p] = make_float4(v[3 * local], v[3 * local + 1], v[3 * local + 2], 0.f);
  vb.gE_row[ws.pos_slot[p]] = (float)ws.sys[b].in.gE;
}

// u_i = d/de G_i(r + e v) (Eqs. 3-5 differentiated along v); one warp per centre
__global__ void __launch_bounds__(kWarps * 32) k_aev_jvp(Ws ws, AevConst ac, VjpBufs vb) {
  extern __shared__ float4 sm4[];
  __shared__ ListHdr hdrs[kWarps];
  const int w = threadIdx.x >> 5;
  const unsigned lane = threadIdx.x & 31;
  const int p = blockIdx.x * kWarps + w;
  if (p >= ws.totals[0]) return;
  // per warp: angular (u, R), (fc, dfc, Rdot, 0), (dv.xyz, 0); radial (R, fc, dfc, Rdot)
  float4* angv = sm4 + (size_t)w * (3 * ws.cap_a + ws.cap_r);
  float4* angf = angv + ws.cap_a;
  float4* angd = angf + ws.cap_a;
  float4* rad = angd + ws.cap_a;
  ListHdr& H = hdrs[w];
  const float4 xi = ws.xyzq[p];
  const float4 vi = vb.v_pos[p];
  const SysDev& d = ws.sys[ws.pos_sys[p]];
  float* U = vb.U + (size_t)ws.pos_slot[p] * ac.Dp;
  load_hdr(ws.nb_cnt + (size_t)p * 16, ac.S, lane, &H);
  const int nr_tot = H.off_r[ac.S], na_tot = H.off_a[ac.S];
  const int* lr = ws.nb_r + (size_t)p * ws.cap_r;
  const int* la = ws.nb_a + (size_t)p * ws.cap_a;
  for (int t = lane; t < nr_tot; t += 32) {
    const int j = lr[t];
    const Geo g = disp(xi, ws.xyzq[j], d);
    const float r = sqrtf(g.dx * g.dx + g.dy * g.dy + g.dz * g.dz);
    const float4 vj = vb.v_pos[j];
    const float rdot = (g.dx * (vj.x - vi.x) + g.dy * (vj.y - vi.y) + g.dz * (vj.z - vi.z)) / r;
    float f, df, ddf;
    fcut3(r, ac.rc_r, &f, &df, &ddf);
    rad[t] = make_float4(r, f, df, rdot);
  }
  for (int t = lane; t < na_tot; t += 32) {
    const int j = la[t];
    const Geo g = disp(xi, ws.xyzq[j], d);
    const float r = sqrtf(g.dx * g.dx + g.dy * g.dy + g.dz * g.dz);
    const float inv = 1.f / r;
    const float4 vj = vb.v_pos[j];
    const float dvx = vj.x - vi.x, dvy = vj.y - vi.y, dvz = vj.z - vi.z;
    float f, df, ddf;
    fcut3(r, ac.rc_a, &f, &df, &ddf);
    angv[t] = make_float4(g.dx * inv, g.dy * inv, g.dz * inv, r);
    angf[t] = make_float4(f, df, (g.dx * dvx + g.dy * dvy + g.dz * dvz) * inv, 0.f);
    angd[t] = make_float4(dvx, dvy, dvz, 0.f);
  }
  __syncwarp();
  // radial: d/de [exp(-eta (R - Rs)^2) f_c(R)] = exp(..) (-2 eta x f_c + f_c') Rdot
  const float cr_ = -ac.eta_r * kLog2e;
  const float my_shf = ac.shf_r[lane & 15];
  const int half = lane >> 4;
  for (int s = 0; s < ac.S; ++s) {
    float acc = 0.f;
    for (int t = H.off_r[s] + half; t < H.off_r[s + 1]; t += 2) {
      const float4 q = rad[t];
      const float x = q.x - my_shf;
      acc = fmaf(fast_exp2(cr_ * x * x) * fmaf(-2.f * ac.eta_r * x, q.y, q.z), q.w, acc);
    }
    acc += __shfl_xor_sync(kFull, acc, 16);
    if (lane < 16) U[ac.rcol[s] + lane] = acc;
  }
  const float ca_ = -ac.eta_a * kLog2e;
  const float m2eta = -2.f * ac.eta_a;
  int pidx = 0;
  for (int s = 0; s < ac.S; ++s)
    for (int u = s; u < ac.S; ++u, ++pidx) {
      const int os = H.off_a[s], cs = H.off_a[s + 1] - os;
      const int ou = H.off_a[u], cu = H.off_a[u + 1] - ou;
      const int same = (s == u);
      const int n_tri = same ? cs * (cs - 1) / 2 : cs * cu;
      float* Ub = U + ac.acol[pidx];
      if (n_tri == 0) {
        Ub[lane] = 0.f;
        continue;
      }
      const float inv_cu = 1.f / (float)max(cu, 1);
      float acc[32];
#pragma unroll
      for (int f = 0; f < 32; ++f) acc[f] = 0.f;
      for (int t0 = 0; t0 < n_tri; t0 += 32) {
        const int t = t0 + lane;
        if (t >= n_tri) continue;
        int j, k;
        decode_pair(t, same, cs, cu, inv_cu, &j, &k);
        const float4 uj = angv[os + j], uk = angv[ou + k];
        const float4 fj = angf[os + j], fk = angf[ou + k];
        const float4 dj = angd[os + j], dk = angd[ou + k];
        const float chat = uj.x * uk.x + uj.y * uk.y + uj.z * uk.z;
        // tangent of cos_hat: (u_k - c u_j).dv_j / R_j + (u_j - c u_k).dv_k / R_k
        const float cdot = ((uk.x - chat * uj.x) * dj.x + (uk.y - chat * uj.y) * dj.y +
                            (uk.z - chat * uj.z) * dj.z) / uj.w +
                           ((uj.x - chat * uk.x) * dk.x + (uj.y - chat * uk.y) * dk.y +
                            (uj.z - chat * uk.z) * dk.z) / uk.w;
        const float c = ac.cos_scale * chat;
        const float cx = uj.y * uk.z - uj.z * uk.y, cy = uj.z * uk.x - uj.x * uk.z,
                    cz = uj.x * uk.y - uj.y * uk.x;
        const float sn = fmaxf(sqrtf(fmaf(1.f - ac.cos_scale * ac.cos_scale, chat * chat,
                                          cx * cx + cy * cy + cz * cz)), 1e-6f);
        const float c_over_s = c / sn;
        const float rb = 0.5f * (uj.w + uk.w);
        const float rbdot = 0.5f * (fj.z + fk.z);
        const float fjk = fj.x * fk.x;
        const float fjkdot = fj.y * fj.z * fk.x + fj.x * fk.y * fk.z;
        const float cpdot = ac.cos_scale * cdot;
        float A[kNA], dA[kNA];
#pragma unroll
        for (int a = 0; a < kNA; ++a) {
          const float x = rb - ac.shf_a[a];
          A[a] = fast_exp2(ca_ * x * x);
          dA[a] = m2eta * x * A[a];
        }
#pragma unroll
        for (int z = 0; z < kNZ; ++z) {
          const float base = fmaf(sn, ac.sin_z[z], fmaf(c, ac.cos_z[z], 1.f));
          const float B1 = ipowf(base, ac.zeta - 1);
          const float B = B1 * base;
          const float dB = (float)ac.zeta * B1 * fmaf(-ac.sin_z[z], c_over_s, ac.cos_z[z]);
#pragma unroll
          for (int a = 0; a < kNA; ++a) {
            const float tdot = dB * cpdot * A[a] * fjk + B * dA[a] * rbdot * fjk + B * A[a] * fjkdot;
            acc[a * kNZ + z] = fmaf(ac.ang_pre, tdot, acc[a * kNZ + z]);
          }
        }
      }
      Ub[lane] = transpose_reduce32(acc, lane);
    }
  for (int f = ac.D + lane; f < ac.Dp; f += 32) U[f] = 0.f;
}


// ---------------------------------------------------------------- dual AEV backward
// Primal: dE/du_e for every edge from dE/dG (as in the force kernel).  Tangent:
// its derivative along (coordinates + e v, dE/dG + e q).  Only the tangent is
// accumulated: d/de F_j = -sum over edges ending at j, d/de F_i = +sum.
__global__ void __launch_bounds__(kWarps * 32) k_aev_bwd_dual(Ws ws, AevConst ac, VjpBufs vb) {
  extern __shared__ float4 sm4[];
  __shared__ ListHdr hdrs[kWarps];
  const int w = threadIdx.x >> 5;
  const unsigned lane = threadIdx.x & 31;
  const int p = blockIdx.x * kWarps + w;
  if (p >= ws.totals[0]) return;
  float4* angv = sm4 + (size_t)w * (4 * ws.cap_a + 64);
  float4* angf = angv + ws.cap_a;     // fc, dfc, ddfc, Rdot
  float4* angd = angf + ws.cap_a;     // dv
  float4* acc3 = angd + ws.cap_a;     // tangent of dE/du per angular neighbour
  float* grad = reinterpret_cast<float*>(acc3 + ws.cap_a);   // radial dE/dG [S*16]
  float* gtan = grad + 128;                                  // radial q [S*16]
  ListHdr& H = hdrs[w];
  const float4 xi = ws.xyzq[p];
  const float4 vi = vb.v_pos[p];
  const SysDev& d = ws.sys[ws.pos_sys[p]];
  const size_t row = (size_t)ws.pos_slot[p] * ac.Dp;
  const float* g_row = ws.dEdG + row;
  const float* q_row = vb.Q + row;
  load_hdr(ws.nb_cnt + (size_t)p * 16, ac.S, lane, &H);
  const int na_tot = H.off_a[ac.S];
  const int* lr = ws.nb_r + (size_t)p * ws.cap_r;
  const int* la = ws.nb_a + (size_t)p * ws.cap_a;
  for (int f = lane; f < ac.S * kNR; f += 32) {   // radial blocks, species by species
    const int c = ac.rcol[f >> 4] + (f & 15);
    grad[f] = g_row[c];
    gtan[f] = q_row[c];
  }
  for (int t = lane; t < na_tot; t += 32) {
    const int j = la[t];
    const Geo g = disp(xi, ws.xyzq[j], d);
    const float r = sqrtf(g.dx * g.dx + g.dy * g.dy + g.dz * g.dz);
    const float inv = 1.f / r;
    const float4 vj = vb.v_pos[j];
    const float dvx = vj.x - vi.x, dvy = vj.y - vi.y, dvz = vj.z - vi.z;
    float f, df, ddf;
    fcut3(r, ac.rc_a, &f, &df, &ddf);
    angv[t] = make_float4(g.dx * inv, g.dy * inv, g.dz * inv, r);
    angf[t] = make_float4(f, df, ddf, (g.dx * dvx + g.dy * dvy + g.dz * dvz) * inv);
    angd[t] = make_float4(dvx, dvy, dvz, 0.f);
    acc3[t] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncwarp();
  float fi[3] = {0.f, 0.f, 0.f};
  // ---- radial edges
  const float cr_ = -ac.eta_r * kLog2e;
  const float eta = ac.eta_r;
  for (int s = 0; s < ac.S; ++s) {
    const float* gs = grad + s * kNR;
    const float* qs = gtan + s * kNR;
    for (int t = H.off_r[s] + lane; t < H.off_r[s + 1]; t += 32) {
      const int j = lr[t];
      const Geo g = disp(xi, ws.xyzq[j], d);
      const float r = sqrtf(g.dx * g.dx + g.dy * g.dy + g.dz * g.dz);
      const float4 vj = vb.v_pos[j];
      const float dvx = vj.x - vi.x, dvy = vj.y - vi.y, dvz = vj.z - vi.z;
      const float ux = g.dx / r, uy = g.dy / r, uz = g.dz / r;
      const float rdot = ux * dvx + uy * dvy + uz * dvz;
      float fc, dfc, ddfc;
      fcut3(r, ac.rc_r, &fc, &dfc, &ddfc);
      float dEdR = 0.f, dEdR_t = 0.f;
#pragma unroll
      for (int rr = 0; rr < kNR; ++rr) {
        const float x = r - ac.shf_r[rr];
        const float e = fast_exp2(cr_ * x * x);
        const float h = fmaf(-2.f * eta * x, fc, dfc);
        const float phi = e * h;
        const float dphi = e * (-2.f * eta * x * h - 2.f * eta * fc - 2.f * eta * x * dfc + ddfc);
        dEdR = fmaf(gs[rr], phi, dEdR);
        dEdR_t = fmaf(qs[rr], phi, fmaf(gs[rr], dphi * rdot, dEdR_t));
      }
      // tangent of dEdR * u with du = (dv - u rdot) / r
      const float sc = dEdR / r;
      const float tx = dEdR_t * ux + sc * (dvx - ux * rdot);
      const float ty = dEdR_t * uy + sc * (dvy - uy * rdot);
      const float tz = dEdR_t * uz + sc * (dvz - uz * rdot);
      atomicAdd(&vb.df_pos[j], make_float4(-tx, -ty, -tz, 0.f));
      fi[0] += tx; fi[1] += ty; fi[2] += tz;
    }
  }
  // ---- angular triplets in dual arithmetic
  const float ca_ = -ac.eta_a * kLog2e;
  const float m2eta = -2.f * ac.eta_a;
  const float kap = ac.cos_scale, one_m_k2 = 1.f - ac.cos_scale * ac.cos_scale;
  int pidx = 0;
  for (int s = 0; s < ac.S; ++s)
    for (int u = s; u < ac.S; ++u, ++pidx) {
      const int os = H.off_a[s], cs = H.off_a[s + 1] - os;
      const int ou = H.off_a[u], cu = H.off_a[u + 1] - ou;
      const int same = (s == u);
      const int n_tri = same ? cs * (cs - 1) / 2 : cs * cu;
      if (n_tri == 0) continue;
      const float inv_cu = 1.f / (float)max(cu, 1);
      const float* gb = g_row + ac.acol[pidx];
      const float* qb = q_row + ac.acol[pidx];
      for (int t0 = 0; t0 < n_tri; t0 += 32) {
        const int t = t0 + lane;
        if (t >= n_tri) continue;
        int jj, kk;
        decode_pair(t, same, cs, cu, inv_cu, &jj, &kk);
        const int tj = os + jj, tk = ou + kk;
        const float4 aj = angv[tj], ak = angv[tk];
        const float4 bj = angf[tj], bk = angf[tk];
        const float4 dj = angd[tj], dk = angd[tk];
        // dual unit vectors, distances and cutoffs
        const Df Rj = dd(aj.w, bj.w), Rk = dd(ak.w, bk.w);
        const Df ujx = dd(aj.x, (dj.x - aj.x * bj.w) / aj.w), ujy = dd(aj.y, (dj.y - aj.y * bj.w) / aj.w),
                 ujz = dd(aj.z, (dj.z - aj.z * bj.w) / aj.w);
        const Df ukx = dd(ak.x, (dk.x - ak.x * bk.w) / ak.w), uky = dd(ak.y, (dk.y - ak.y * bk.w) / ak.w),
                 ukz = dd(ak.z, (dk.z - ak.z * bk.w) / ak.w);
        const Df fj = dd(bj.x, bj.y * bj.w), fk = dd(bk.x, bk.y * bk.w);
        const Df dfj = dd(bj.y, bj.z * bj.w), dfk = dd(bk.y, bk.z * bk.w);
        const Df chat = ujx * ukx + ujy * uky + ujz * ukz;
        const Df c = kap * chat;
        const Df crx = ujy * ukz - ujz * uky, cry = ujz * ukx - ujx * ukz, crz = ujx * uky - ujy * ukx;
        Df sn = dsqrt(crx * crx + cry * cry + crz * crz + one_m_k2 * (chat * chat));
        if (sn.v < 1e-6f) sn = dd(1e-6f, 0.f);
        const Df cos_ = c / sn;
        const Df rb = 0.5f * (Rj + Rk);
        Df A[kNA], dA[kNA];
#pragma unroll
        for (int a = 0; a < kNA; ++a) {
          const Df x = rb - dd(ac.shf_a[a]);
          A[a] = dexp2(ca_ * (x * x));
          dA[a] = (m2eta * x) * A[a];
        }
        Df tc = dd(0.f), tR = dd(0.f), tf = dd(0.f);
#pragma unroll
        for (int z = 0; z < kNZ; ++z) {
          const Df base = dd(1.f) + ac.cos_z[z] * c + ac.sin_z[z] * sn;
          const float b1 = ipowf(base.v, ac.zeta - 1);
          const float b2 = ac.zeta > 1 ? ipowf(base.v, ac.zeta - 2) : 0.f;
          const Df B1 = dd(b1, (float)(ac.zeta - 1) * b2 * base.d);
          const Df B = B1 * base;
          const Df dB = B1 * (dd(ac.cos_z[z]) - ac.sin_z[z] * cos_);
          Df P = dd(0.f), Q = dd(0.f);
#pragma unroll
          for (int a = 0; a < kNA; ++a) {
            const Df G = dd(gb[a * kNZ + z], qb[a * kNZ + z]);
            P = P + G * A[a];
            Q = Q + G * dA[a];
          }
          tc = tc + dB * P;
          tR = tR + B * Q;
          tf = tf + B * P;
        }
        const Df fjk = fj * fk;
        tc = (ac.ang_pre * (float)ac.zeta) * (tc * fjk);
        tR = ac.ang_pre * (tR * fjk);
        tf = ac.ang_pre * tf;
        const Df dEdchat = kap * tc;
        const Df sj = dEdchat / Rj, sk = dEdchat / Rk;
        const Df rj = 0.5f * tR + tf * (dfj * fk);
        const Df rk = 0.5f * tR + tf * (fj * dfk);
        const Df gux = sj * (ukx - chat * ujx) + rj * ujx, guy = sj * (uky - chat * ujy) + rj * ujy,
                 guz = sj * (ukz - chat * ujz) + rj * ujz;
        const Df gvx = sk * (ujx - chat * ukx) + rk * ukx, gvy = sk * (ujy - chat * uky) + rk * uky,
                 gvz = sk * (ujz - chat * ukz) + rk * ukz;
        atomicAdd(&acc3[tj].x, gux.d);
        atomicAdd(&acc3[tj].y, guy.d);
        atomicAdd(&acc3[tj].z, guz.d);
        atomicAdd(&acc3[tk].x, gvx.d);
        atomicAdd(&acc3[tk].y, gvy.d);
        atomicAdd(&acc3[tk].z, gvz.d);
      }
    }
  __syncwarp();
  for (int t = lane; t < na_tot; t += 32) {
    const float4 a = acc3[t];
    atomicAdd(&vb.df_pos[la[t]], make_float4(-a.x, -a.y, -a.z, 0.f));
    fi[0] += a.x; fi[1] += a.y; fi[2] += a.z;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fi[0] += __shfl_xor_sync(kFull, fi[0], o);
    fi[1] += __shfl_xor_sync(kFull, fi[1], o);
    fi[2] += __shfl_xor_sync(kFull, fi[2], o);
  }
  if (lane == 0) atomicAdd(&vb.df_pos[p], make_float4(fi[0], fi[1], fi[2], 0.f));
}

// CELU'' from the stored CELU' (z <= 0: CELU' = exp(z/alpha), CELU'' = CELU'/alpha;
// z > 0: CELU' = 1, CELU'' = 0)
__device__ __forceinline__ float celu_dd(float dz, float inv_alpha) {
  return dz < 1.f ? dz * inv_alpha : 0.f;
}

// per (row, member): e = h3 . w4, delta3 = w4 CELU'(z3), delta3' = w4 CELU''(z3) z3'
__global__ void k_vjp_out3(Ws ws, VjpBufs vb, const float* w4, int S, int E, int h3, float inv_alpha) {
  const int total = ws.seg_start[S];
  const long long n = (long long)total * E;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(q / E), e = (int)(q % E);
    int s = 0;
    while (s + 1 < S && m >= ws.seg_start[s + 1]) ++s;
    const float* wv = w4 + ((size_t)e * S + s) * h3;
    const size_t o = (size_t)m * E * h3 + (size_t)e * h3;
    float dot = 0.f;
    for (int k = 0; k < h3; ++k) {
      const float D = vb.D3[o + k];
      dot = fmaf(vb.H3[o + k], wv[k], dot);
      vb.dl3[o + k] = wv[k] * D;
      vb.dl3d[o + k] = wv[k] * celu_dd(D, inv_alpha) * vb.Z3d[o + k];
    }
    vb.e_row[(size_t)e * ws.row_cap + m] = dot;
  }
}

// delta = Ah * D ; delta' = Ah * CELU'' * Z' + Az * D   (element-wise, [rows][E*h])
__global__ void k_vjp_delta(const int* seg_start, int S, int width, const float* Ah, const float* Az,
                            const float* D, const float* Zd, float* dl, float* dld, float inv_alpha) {
  const long long n = (long long)seg_start[S] * width;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float a = Ah[i], dz = D[i];
    dl[i] = a * dz;
    dld[i] = a * celu_dd(dz, inv_alpha) * Zd[i] + Az[i] * dz;
  }
}

// per-species weight/bias gradients of one layer, summed over the species' rows:
//   C[o][k] = scale * sum_m [X1[m,o] (gE_m Y1[m,k] - Y2[m,k]) - X2[m,o] Y1[m,k]]
//   (k == n_in: bias column with Y1 = 1, Y2 = 0); written to the flat layout
__global__ void __launch_bounds__(256) k_wgrad(WgradArgs a, const int* seg_start, const int* counts,
                                               const float* gE_row) {
  __shared__ float sx1[32][33], sx2[32][33], sy1[32][33], sy2[32][33], sg[32];
  const int es = blockIdx.z, e = es / a.S, s = es % a.S;
  const int o0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  const int beg = seg_start[s], end = seg_start[s] + counts[s];
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int m0 = beg; m0 < end; m0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const int m = m0 + r;
      const bool ok = m < end;
      const int o = o0 + tx, k = k0 + tx;
      sx1[r][tx] = (ok && o < a.n_out) ? a.X1[(size_t)m * a.ldx + (size_t)e * a.x_net + o] : 0.f;
      sx2[r][tx] = (ok && o < a.n_out) ? a.X2[(size_t)m * a.ldx + (size_t)e * a.x_net + o] : 0.f;
      float y1 = 0.f, y2 = 0.f;
      if (ok) {
        if (k < a.n_in) {
          y1 = a.Y1[(size_t)m * a.ldy + (size_t)e * a.y_net + k];
          y2 = a.Y2[(size_t)m * a.ldy + (size_t)e * a.y_net + k];
        } else if (k == a.n_in) {
          y1 = 1.f;
        }
      }
      sy1[r][tx] = y1;
      sy2[r][tx] = y2;
      if (ty == 0) sg[tx] = (m0 + tx < end) ? gE_row[m0 + tx] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
      const float y1 = sy1[r][tx], y2 = sy2[r][tx];
      const float gy = fmaf(sg[r], y1, -y2);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int oo = ty + 8 * i;
        acc[i] = fmaf(sx1[r][oo], gy, fmaf(-sx2[r][oo], y1, acc[i]));
      }
    }
    __syncthreads();
  }
  const int k = k0 + tx;
  float* base = a.out + ((size_t)e * a.S + s) * a.per_net + a.layer_off;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int o = o0 + ty + 8 * i;
    if (o >= a.n_out) continue;
    if (k < a.n_in_real)
      base[(size_t)o * a.n_in_real + (a.feat_of_col ? a.feat_of_col[k] : k)] = a.scale * acc[i];
    else if (k == a.n_in) base[(size_t)a.n_out * a.n_in_real + o] = a.scale * acc[i];
  }
}

// output layer: dw4[k] = scale sum_m (gE_m H3[m,k] - H3'[m,k]); db4 = scale sum_m gE_m
__global__ void k_wgrad_out(VjpBufs vb, const int* seg_start, const int* counts, int S, int E, int h3,
                            float scale, float* out, long long per_net, long long off4) {
  const int es = blockIdx.x, e = es / S, s = es % S;
  const int beg = seg_start[s], end = seg_start[s] + counts[s];
  float* base = out + ((size_t)e * S + s) * per_net + off4;
  for (int k = threadIdx.x; k <= h3; k += blockDim.x) {
    float acc = 0.f;
    for (int m = beg; m < end; ++m) {
      const float g = vb.gE_row[m];
      if (k < h3) {
        const size_t o = (size_t)m * E * h3 + (size_t)e * h3 + k;
        acc += g * vb.H3[o] - vb.H3d[o];
      } else {
        acc += g;
      }
    }
    base[k] = scale * acc;   // k == h3 is the output bias
  }
}

// dL/dr = d/de F - gE F, in the caller's atom order (zero outside the mask)
__global__ void k_vjp_scatter(Ws ws, VjpBufs vb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ws.totals[0]) return;
  const int b = ws.pos_sys[p];
  const SysDev& d = ws.sys[b];
  const int local = ws.pos_src[p] - d.in.in_base;
  const float4 df = vb.df_pos[p], f = ws.f_pos[p];
  const float g = (float)d.in.gE;
  float* out = d.in.dLdR + 3 * (size_t)local;
  out[0] = df.x - g * f.x;
  out[1] = df.y - g * f.y;
  out[2] = df.z - g * f.z;
}

// zero the packed tangent accumulators
__global__ void k_vjp_zero(VjpBufs vb, int n_in) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_in) vb.df_pos[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

}  // namespace

size_t vjp_jvp_smem(const Ws& ws) { return (size_t)kWarps * (3 * ws.cap_a + ws.cap_r) * sizeof(float4); }
size_t vjp_dual_smem(const Ws& ws) { return (size_t)kWarps * (4 * ws.cap_a + 64) * sizeof(float4); }

// raise (never lower) the kernels' dynamic shared-memory limits: other handles
// of the process may need larger ones
cudaError_t vjp_set_smem(const Ws& ws) {
  const void* fn[2] = {(const void*)k_aev_jvp, (const void*)k_aev_bwd_dual};
  const int need[2] = {(int)vjp_jvp_smem(ws), (int)vjp_dual_smem(ws)};
  for (int i = 0; i < 2; ++i) {
    cudaFuncAttributes attr;
    cudaError_t e = cudaFuncGetAttributes(&attr, fn[i]);
    if (e != cudaSuccess) return e;
    if (attr.maxDynamicSharedSizeBytes < need[i]) {
      e = cudaFuncSetAttribute(fn[i], cudaFuncAttributeMaxDynamicSharedMemorySize, need[i]);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

void launch_vjp_zero(const Ws& ws, const VjpBufs& vb, int n_in, cudaStream_t st) {
  (void)ws;
  k_vjp_zero<<<(n_in + 255) / 256, 256, 0, st>>>(vb, n_in);
}
void launch_gather_v(const Ws& ws, const VjpBufs& vb, int n_in, cudaStream_t st) {
  k_gather_v<<<(n_in + 255) / 256, 256, 0, st>>>(ws, vb);
}
void launch_aev_jvp(const Ws& ws, const AevConst& ac, const VjpBufs& vb, int n_in, cudaStream_t st) {
  k_aev_jvp<<<(n_in + kWarps - 1) / kWarps, kWarps * 32, vjp_jvp_smem(ws), st>>>(ws, ac, vb);
}
void launch_aev_bwd_dual(const Ws& ws, const AevConst& ac, const VjpBufs& vb, int n_in, cudaStream_t st) {
  k_aev_bwd_dual<<<(n_in + kWarps - 1) / kWarps, kWarps * 32, vjp_dual_smem(ws), st>>>(ws, ac, vb);
}
void launch_vjp_out3(const Ws& ws, const VjpBufs& vb, const float* w4, int S, int E, int h3, float alpha,
                     cudaStream_t st) {
  k_vjp_out3<<<4 * 152, 256, 0, st>>>(ws, vb, w4, S, E, h3, 1.f / alpha);
}
void launch_vjp_delta(const Ws& ws, int S, int width, const float* Ah, const float* Az, const float* D,
                      const float* Zd, float* dl, float* dld, float alpha, cudaStream_t st) {
  k_vjp_delta<<<4 * 152, 256, 0, st>>>(ws.seg_start, S, width, Ah, Az, D, Zd, dl, dld, 1.f / alpha);
}
void launch_wgrad(const WgradArgs& a, const Ws& ws, const VjpBufs& vb, int E, cudaStream_t st) {
  dim3 grid((a.n_in + 1 + 31) / 32, (a.n_out + 31) / 32, E * a.S);
  k_wgrad<<<grid, 256, 0, st>>>(a, ws.seg_start, ws.species_count, vb.gE_row);
}
void launch_wgrad_out(const Ws& ws, const VjpBufs& vb, int S, int E, int h3, float* out, long long per_net,
                      long long off4, cudaStream_t st) {
  k_wgrad_out<<<E * S, 128, 0, st>>>(vb, ws.seg_start, ws.species_count, S, E, h3, 1.f / E, out, per_net, off4);
}
void launch_vjp_scatter(const Ws& ws, const VjpBufs& vb, int n_in, cudaStream_t st) {
  k_vjp_scatter<<<(n_in + 255) / 256, 256, 0, st>>>(ws, vb);
}

}  // namespace nnp
