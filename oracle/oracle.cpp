// FP64 CPU oracle for the ANI-style neural-network potential of the Deep-HP
// paper (arXiv 2207.14276, Sec. "Neural Network Potentials" / "ANI models").
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow definition of what
// the GPU library computes.  Only the test-suite, the package smoke check and
// the benchmark's CPU-baseline leg may load it.  It shares no code, header,
// table or helper with the CUDA library.
//
// Everything is written straight from the paper's equations, in double
// precision, with no blocking, fusion or reordering:
//   Eq. 2  E_T = sum_i E_i(G_i)                      (energy decomposition)
//   Eq. 3  f_c(R) = 0.5 cos(pi R / Rc) + 0.5, R <= Rc; 0 beyond
//   Eq. 4  G^rad_{i,m} = sum_{j != i, R_ij <= Rc} exp(-eta (R_ij - R_s)^2) f_c(R_ij)
//   Eq. 5  G^ang_{i,m} = 2^(1-zeta) sum_{j,k != i}
//              (1 + cos(theta_ijk - theta_s))^zeta
//              exp(-eta ((R_ij + R_ik)/2 - R_s)^2) f_c(R_ij) f_c(R_ik)
//          with one radial sub-AEV per species and one angular sub-AEV per
//          unordered species pair (N radial + N(N+1)/2 angular blocks).
//   Eq. 7  hybrid potential: only the masked (solute) region P enters V_ML(P).
// Readings where the paper is silent (each is a plain data choice):
//   * the angular sum runs over unordered pairs j < k (j = k excluded) with the
//     printed 2^(1-zeta) prefactor;
//   * the angular cutoff radius is its own parameter (rc_a), radial is rc_r;
//   * theta_ijk = acos(cos_scale * cos_angle) with cos_scale = 1 by default;
//   * radial block s*n_r + r first, then angular block p(s,t) (s <= t, upper
//     triangle in row-major order), inside a block index a*n_z + z;
//   * each species has one feed-forward network per ensemble member
//     (activation CELU, alpha given), the ensemble energy is the mean;
//   * periodic boxes are orthorhombic with the minimum-image convention;
//   * atoms outside the mask are neither centres nor neighbours and get zero
//     force.
// Forces are the analytic chain rule F = -dE/dr written out by hand.  The
// force-matching gradient uses a forward-mode dual number along the
// coordinate direction v = dL/dF, run through the same templated code.
// Pins (CPU tests): hand-derived AEV values at special geometries (the golden
// fixture of Eqs. 3-5), the networks against a numpy chain, invariants
// (translation, rotation, permutation, zero net force and torque, extensivity,
// the mask), and finite differences of the energy and of the force-matching
// loss.  Parity unpinned: the absolute energies of the synthetic models (the
// paper prints no worked example with its weights).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// ---------------------------------------------------------------- dual number
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
inline Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
inline Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
inline Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual exp(Dual a) { double e = std::exp(a.v); return Dual(e, e * a.d); }
inline Dual cos(Dual a) { return Dual(std::cos(a.v), -std::sin(a.v) * a.d); }
inline Dual sin(Dual a) { return Dual(std::sin(a.v), std::cos(a.v) * a.d); }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2 * s)); }
inline Dual acos(Dual a) { return Dual(std::acos(a.v), -a.d / std::sqrt(1 - a.v * a.v)); }
inline Dual pow(Dual a, double p) {
  return Dual(std::pow(a.v, p), p * std::pow(a.v, p - 1) * a.d);
}
inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
using std::exp; using std::cos; using std::sin; using std::sqrt; using std::acos; using std::pow;

template <class T> inline T sq(T x) { return x * x; }

// ---------------------------------------------------------------- model
struct Model {
  int S = 0;
  double rc_r = 0, eta_r = 0, rc_a = 0, eta_a = 0, zeta = 0, cos_scale = 1;
  std::vector<double> shf_r, shf_a, shf_z;
  int n_ens = 1, n_layers = 0;
  std::vector<int> widths;
  std::vector<double> flat;      // weights in the flat layout (see synth/params.py)
  std::vector<size_t> w_ofs;     // offset of W for (e, s, l)
  std::vector<double> shift;     // per-species energy shift
  double alpha = 0.1;

  int nr() const { return (int)shf_r.size(); }
  int na() const { return (int)shf_a.size(); }
  int nz() const { return (int)shf_z.size(); }
  int D() const { return S * nr() + S * (S + 1) / 2 * na() * nz(); }
  size_t idx(int e, int s, int l) const { return ((size_t)e * S + s) * n_layers + l; }
  const double* W(int e, int s, int l) const { return flat.data() + w_ofs[idx(e, s, l)]; }
  const double* b(int e, int s, int l) const {
    return W(e, s, l) + (size_t)widths[l + 1] * widths[l];
  }
  // angular block of the unordered species pair {s, t} (upper triangle, row-major)
  int pair_block(int s, int t) const {
    if (s > t) std::swap(s, t);
    int p = 0;
    for (int u = 0; u < s; ++u) p += S - u;
    return p + (t - s);
  }
};

// ---------------------------------------------------------------- Eq. 3
template <class T> T fcut(T R, double rc) {
  if (val(R) > rc) return T(0.0);
  return 0.5 * cos(M_PI * R / rc) + 0.5;
}
template <class T> T fcut_deriv(T R, double rc) {
  if (val(R) > rc) return T(0.0);
  return -0.5 * (M_PI / rc) * sin(M_PI * R / rc);
}
template <class T> T celu(T z, double alpha) {
  if (val(z) > 0) return z;
  return alpha * (exp(z / alpha) - 1.0);
}
template <class T> T celu_grad(T z, double alpha) {
  if (val(z) > 0) return T(1.0);
  return exp(z / alpha);
}

// ---------------------------------------------------------------- neighbours
template <class T> struct Nb { int j; T d[3]; T R; };

// minimum-image displacement r_j - r_i (orthorhombic box, or plain if box == NULL)
template <class T>
void displacement(const T* xyz, int i, int j, const double* box, T d[3]) {
  for (int c = 0; c < 3; ++c) {
    d[c] = xyz[3 * j + c] - xyz[3 * i + c];
    if (box) d[c] = d[c] - box[c] * std::nearbyint(val(d[c]) / box[c]);
  }
}

// all j != i inside the mask with R_ij <= rc, by brute force over every atom
template <class T>
std::vector<Nb<T>> neighbours_of(int i, int n, const T* xyz, const double* box,
                                 const uint8_t* mask, double rc) {
  std::vector<Nb<T>> out;
  for (int j = 0; j < n; ++j) {
    if (j == i || (mask && !mask[j])) continue;
    Nb<T> q;
    q.j = j;
    displacement(xyz, i, j, box, q.d);
    T R2 = q.d[0] * q.d[0] + q.d[1] * q.d[1] + q.d[2] * q.d[2];
    if (val(R2) <= rc * rc) {
      q.R = sqrt(R2);
      out.push_back(q);
    }
  }
  return out;
}

template <class T> T clamp_unit(T x) {
  if (val(x) > 1.0) return T(1.0);
  if (val(x) < -1.0) return T(-1.0);
  return x;
}

// ---------------------------------------------------------------- Eqs. 4, 5
template <class T>
void aev_centre(const Model& m, const std::vector<Nb<T>>& nb, const uint8_t* sp, T* G) {
  const int D = m.D(), nr = m.nr(), na = m.na(), nz = m.nz();
  for (int f = 0; f < D; ++f) G[f] = T(0.0);
  // Eq. 4: radial Gaussians times the cosine cutoff, one block per neighbour species
  for (const auto& q : nb) {
    if (val(q.R) > m.rc_r) continue;
    T fc = fcut(q.R, m.rc_r);
    for (int r = 0; r < nr; ++r)
      G[sp[q.j] * nr + r] += exp(-m.eta_r * sq(q.R - m.shf_r[r])) * fc;
  }
  // Eq. 5: angular terms over unordered neighbour pairs inside rc_a
  std::vector<const Nb<T>*> an;
  for (const auto& q : nb)
    if (val(q.R) <= m.rc_a) an.push_back(&q);
  const double pre = std::pow(2.0, 1.0 - m.zeta);
  for (size_t a = 0; a < an.size(); ++a)
    for (size_t b = a + 1; b < an.size(); ++b) {
      const Nb<T>& qj = *an[a];
      const Nb<T>& qk = *an[b];
      T cosang = (qj.d[0] * qk.d[0] + qj.d[1] * qk.d[1] + qj.d[2] * qk.d[2]) / (qj.R * qk.R);
      T theta = acos(clamp_unit(m.cos_scale * cosang));
      T fcjk = fcut(qj.R, m.rc_a) * fcut(qk.R, m.rc_a);
      T Rbar = (qj.R + qk.R) / 2.0;
      int base = m.S * nr + m.pair_block(sp[qj.j], sp[qk.j]) * na * nz;
      for (int ia = 0; ia < na; ++ia) {
        T rad = exp(-m.eta_a * sq(Rbar - m.shf_a[ia]));
        for (int iz = 0; iz < nz; ++iz)
          G[base + ia * nz + iz] += pre * pow(1.0 + cos(theta - m.shf_z[iz]), m.zeta) * rad * fcjk;
      }
    }
}

// ---------------------------------------------------------------- the networks
template <class T> struct Tape { std::vector<std::vector<T>> z, h; };

// one per-species network, layer l: z = W h + b, h' = CELU(z) (identity on the output)
template <class T>
T mlp_forward(const Model& m, int e, int s, const T* G, Tape<T>& tp) {
  const int L = m.n_layers;
  tp.z.assign(L + 1, {});
  tp.h.assign(L + 1, {});
  tp.h[0].assign(G, G + m.widths[0]);
  for (int l = 0; l < L; ++l) {
    const int n_in = m.widths[l], n_out = m.widths[l + 1];
    const double* W = m.W(e, s, l);
    const double* b = m.b(e, s, l);
    tp.z[l + 1].assign(n_out, T(0.0));
    tp.h[l + 1].assign(n_out, T(0.0));
    for (int o = 0; o < n_out; ++o) {
      T acc = T(b[o]);
      for (int k = 0; k < n_in; ++k) acc += W[(size_t)o * n_in + k] * tp.h[l][k];
      tp.z[l + 1][o] = acc;
      tp.h[l + 1][o] = (l + 1 < L) ? celu(acc, m.alpha) : acc;
    }
  }
  return tp.h[L][0];
}

// reverse pass: dG += scale * d(out)/dG ; dW (flat layout) += scale * d(out)/dW
template <class T>
void mlp_backward(const Model& m, int e, int s, const Tape<T>& tp, double scale, T* dG, T* dW) {
  const int L = m.n_layers;
  std::vector<T> delta(1, T(scale));  // d out / d z_L
  for (int l = L - 1; l >= 0; --l) {
    const int n_in = m.widths[l], n_out = m.widths[l + 1];
    const double* W = m.W(e, s, l);
    if (dW) {
      T* gW = dW + m.w_ofs[m.idx(e, s, l)];
      T* gb = gW + (size_t)n_out * n_in;
      for (int o = 0; o < n_out; ++o) {
        for (int k = 0; k < n_in; ++k) gW[(size_t)o * n_in + k] += delta[o] * tp.h[l][k];
        gb[o] += delta[o];
      }
    }
    std::vector<T> g(n_in, T(0.0));
    for (int o = 0; o < n_out; ++o)
      for (int k = 0; k < n_in; ++k) g[k] += W[(size_t)o * n_in + k] * delta[o];
    if (l > 0) {
      for (int k = 0; k < n_in; ++k) g[k] = g[k] * celu_grad(tp.z[l][k], m.alpha);
      delta = g;
    } else {
      for (int k = 0; k < n_in; ++k) dG[k] += g[k];
    }
  }
}

// ---------------------------------------------------------------- d AEV / d r
// adds dE/du (u = r_j - r_i) to atom j and subtracts it from atom i; virial
// W -= u (x) dE/du
template <class T>
void add_edge(int i, int j, const T u[3], const T g[3], T* dEdx, T* vir) {
  for (int c = 0; c < 3; ++c) {
    dEdx[3 * j + c] += g[c];
    dEdx[3 * i + c] -= g[c];
  }
  if (vir)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) vir[3 * a + b] -= u[a] * g[b];
}

// chain rule of Eqs. 3-5: given dE/dG_i, accumulate dE/dr for i and its neighbours
template <class T>
void aev_backward_centre(const Model& m, int i, const std::vector<Nb<T>>& nb, const uint8_t* sp,
                         const T* dG, T* dEdx, T* vir) {
  const int nr = m.nr(), na = m.na(), nz = m.nz();
  for (const auto& q : nb) {
    if (val(q.R) > m.rc_r) continue;
    T fc = fcut(q.R, m.rc_r), dfc = fcut_deriv(q.R, m.rc_r);
    T dEdR = T(0.0);
    for (int r = 0; r < nr; ++r) {
      T gauss = exp(-m.eta_r * sq(q.R - m.shf_r[r]));
      T dgauss = gauss * (-2.0 * m.eta_r) * (q.R - m.shf_r[r]);
      dEdR += dG[sp[q.j] * nr + r] * (dgauss * fc + gauss * dfc);
    }
    T g[3];
    for (int c = 0; c < 3; ++c) g[c] = dEdR * q.d[c] / q.R;
    add_edge(i, q.j, q.d, g, dEdx, vir);
  }
  std::vector<const Nb<T>*> an;
  for (const auto& q : nb)
    if (val(q.R) <= m.rc_a) an.push_back(&q);
  const double pre = std::pow(2.0, 1.0 - m.zeta);
  for (size_t a = 0; a < an.size(); ++a)
    for (size_t b = a + 1; b < an.size(); ++b) {
      const Nb<T>& qj = *an[a];
      const Nb<T>& qk = *an[b];
      const T Rj = qj.R, Rk = qk.R;
      T cosang = (qj.d[0] * qk.d[0] + qj.d[1] * qk.d[1] + qj.d[2] * qk.d[2]) / (Rj * Rk);
      T x = clamp_unit(m.cos_scale * cosang);
      T theta = acos(x);
      T dtheta_dcos = -m.cos_scale / sqrt(1.0 - x * x);
      T fj = fcut(Rj, m.rc_a), fk = fcut(Rk, m.rc_a);
      T dfj = fcut_deriv(Rj, m.rc_a), dfk = fcut_deriv(Rk, m.rc_a);
      T Rbar = (Rj + Rk) / 2.0;
      int base = m.S * nr + m.pair_block(sp[qj.j], sp[qk.j]) * na * nz;
      T dE_dtheta = T(0.0), dE_dRj = T(0.0), dE_dRk = T(0.0);
      for (int ia = 0; ia < na; ++ia) {
        T rad = exp(-m.eta_a * sq(Rbar - m.shf_a[ia]));
        T drad = rad * (-2.0 * m.eta_a) * (Rbar - m.shf_a[ia]);  // d rad / d Rbar
        for (int iz = 0; iz < nz; ++iz) {
          T c1 = 1.0 + cos(theta - m.shf_z[iz]);
          T ang = pre * pow(c1, m.zeta);
          T dang = pre * m.zeta * pow(c1, m.zeta - 1.0) * (-1.0 * sin(theta - m.shf_z[iz]));
          T gz = dG[base + ia * nz + iz];
          dE_dtheta += gz * dang * rad * fj * fk;
          dE_dRj += gz * ang * (0.5 * drad * fj * fk + rad * dfj * fk);
          dE_dRk += gz * ang * (0.5 * drad * fj * fk + rad * fj * dfk);
        }
      }
      T gu[3], gv[3];
      for (int c = 0; c < 3; ++c) {
        T dcos_du = qk.d[c] / (Rj * Rk) - cosang * qj.d[c] / (Rj * Rj);
        T dcos_dv = qj.d[c] / (Rj * Rk) - cosang * qk.d[c] / (Rk * Rk);
        gu[c] = dE_dtheta * dtheta_dcos * dcos_du + dE_dRj * qj.d[c] / Rj;
        gv[c] = dE_dtheta * dtheta_dcos * dcos_dv + dE_dRk * qk.d[c] / Rk;
      }
      add_edge(i, qj.j, qj.d, gu, dEdx, vir);
      add_edge(i, qk.j, qk.d, gv, dEdx, vir);
    }
}

// ---------------------------------------------------------------- Eq. 2
// E = sum_i [ mean_e net_{e,s_i}(G_i) + shift_{s_i} ] over the atoms in the mask
template <class T>
T energy_forces(const Model& m, int n, const T* xyz, const uint8_t* sp, const double* box,
                const uint8_t* mask, T* forces, T* vir, T* atom_e, T* aev_out, T* dEdG_out, T* dEdW,
                const int32_t* centres = nullptr, int n_centres = -1) {
  const int D = m.D();
  const double rc = std::max(m.rc_r, m.rc_a);
  std::vector<T> dEdx(3 * (size_t)n, T(0.0)), G(D), dG(D);
  if (vir)
    for (int k = 0; k < 9; ++k) vir[k] = T(0.0);
  T E = T(0.0);
  Tape<T> tp;
  if (atom_e)
    for (int i = 0; i < n; ++i) atom_e[i] = T(0.0);
  const int n_loop = centres ? n_centres : n;
  for (int t = 0; t < n_loop; ++t) {
    const int i = centres ? centres[t] : t;
    if (mask && !mask[i]) continue;
    auto nb = neighbours_of(i, n, xyz, box, mask, rc);
    aev_centre(m, nb, sp, G.data());
    for (int f = 0; f < D; ++f) dG[f] = T(0.0);
    T Ei = T(m.shift[sp[i]]);
    for (int e = 0; e < m.n_ens; ++e) {
      Ei += mlp_forward(m, e, sp[i], G.data(), tp) / (double)m.n_ens;
      mlp_backward(m, e, sp[i], tp, 1.0 / m.n_ens, dG.data(), dEdW);
    }
    E += Ei;
    if (atom_e) atom_e[i] = Ei;
    if (aev_out)
      for (int f = 0; f < D; ++f) aev_out[(size_t)i * D + f] = G[f];
    if (dEdG_out)
      for (int f = 0; f < D; ++f) dEdG_out[(size_t)i * D + f] = dG[f];
    aev_backward_centre(m, i, nb, sp, dG.data(), dEdx.data(), vir);
  }
  if (forces)
    for (size_t k = 0; k < 3 * (size_t)n; ++k) forces[k] = -1.0 * dEdx[k];
  return E;
}

// ---------------------------------------------------------------- cell list
// A second, independent neighbour search (linked cells) used only to check the
// brute-force list: identical pair sets are expected.
int64_t neighbours_cells(int n, const double* xyz, const double* box, const uint8_t* mask,
                         double rc, int64_t cap, int32_t* out) {
  double lo[3], len[3];
  int nc[3];
  for (int c = 0; c < 3; ++c) {
    if (box) {
      lo[c] = 0;
      len[c] = box[c];
    } else {
      double a = 1e300, b = -1e300;
      for (int i = 0; i < n; ++i) {
        a = std::min(a, xyz[3 * i + c]);
        b = std::max(b, xyz[3 * i + c]);
      }
      if (n == 0) a = b = 0;
      lo[c] = a;
      len[c] = (b - a) + 1e-9;
    }
    nc[c] = std::max(1, (int)std::floor(len[c] / rc));
  }
  auto cell_of = [&](int i, int cc[3]) {
    for (int c = 0; c < 3; ++c) {
      double x = xyz[3 * i + c] - lo[c];
      if (box) x -= box[c] * std::floor(x / box[c]);
      int k = (int)std::floor(x / len[c] * nc[c]);
      cc[c] = std::min(std::max(k, 0), nc[c] - 1);
    }
  };
  std::vector<std::vector<int>> cells((size_t)nc[0] * nc[1] * nc[2]);
  for (int i = 0; i < n; ++i) {
    if (mask && !mask[i]) continue;
    int cc[3];
    cell_of(i, cc);
    cells[((size_t)cc[0] * nc[1] + cc[1]) * nc[2] + cc[2]].push_back(i);
  }
  int64_t cnt = 0;
  for (int i = 0; i < n; ++i) {
    if (mask && !mask[i]) continue;
    int cc[3];
    cell_of(i, cc);
    std::vector<size_t> visit;
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          int k[3] = {cc[0] + dx, cc[1] + dy, cc[2] + dz};
          bool ok = true;
          for (int c = 0; c < 3; ++c) {
            if (box) k[c] = ((k[c] % nc[c]) + nc[c]) % nc[c];
            else if (k[c] < 0 || k[c] >= nc[c]) ok = false;
          }
          if (ok) visit.push_back(((size_t)k[0] * nc[1] + k[1]) * nc[2] + k[2]);
        }
    std::sort(visit.begin(), visit.end());
    visit.erase(std::unique(visit.begin(), visit.end()), visit.end());
    for (size_t cell : visit)
      for (int j : cells[cell]) {
        if (j == i) continue;
        double d[3];
        displacement(xyz, i, j, box, d);
        if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] <= rc * rc) {
          if (cnt < cap) {
            out[2 * cnt] = i;
            out[2 * cnt + 1] = j;
          }
          ++cnt;
        }
      }
  }
  return cnt;
}

}  // namespace

// ================================================================ C entry points
extern "C" {

void* oracle_model_new(int S, double rc_r, double eta_r, int n_shf_r, const double* shf_r,
                       double rc_a, double eta_a, double zeta, int n_shf_a, const double* shf_a,
                       int n_shf_z, const double* shf_z, double cos_scale, int n_ens, int n_layers,
                       const int* widths, const double* weights, const double* shift,
                       double alpha) {
  Model* m = new Model;
  m->S = S;
  m->rc_r = rc_r; m->eta_r = eta_r; m->rc_a = rc_a; m->eta_a = eta_a;
  m->zeta = zeta; m->cos_scale = cos_scale; m->alpha = alpha;
  m->shf_r.assign(shf_r, shf_r + n_shf_r);
  m->shf_a.assign(shf_a, shf_a + n_shf_a);
  m->shf_z.assign(shf_z, shf_z + n_shf_z);
  m->n_ens = n_ens;
  m->n_layers = n_layers;
  m->widths.assign(widths, widths + n_layers + 1);
  size_t ofs = 0;
  m->w_ofs.assign((size_t)n_ens * S * n_layers, 0);
  for (int e = 0; e < n_ens; ++e)
    for (int s = 0; s < S; ++s)
      for (int l = 0; l < n_layers; ++l) {
        m->w_ofs[m->idx(e, s, l)] = ofs;
        ofs += (size_t)widths[l + 1] * widths[l] + widths[l + 1];
      }
  m->flat.assign(weights, weights + ofs);
  m->shift.assign(S, 0.0);
  if (shift)
    for (int s = 0; s < S; ++s) m->shift[s] = shift[s];
  return m;
}

void oracle_model_free(void* m) { delete static_cast<Model*>(m); }
int oracle_aev_dim(void* m) { return static_cast<Model*>(m)->D(); }
int64_t oracle_n_weights(void* m) { return (int64_t) static_cast<Model*>(m)->flat.size(); }

// brute-force O(N^2) neighbour pairs (i, j), i != j, R_ij <= rc; returns the count
int64_t oracle_neighbours_brute(int n, const double* xyz, const double* box, const uint8_t* mask,
                                double rc, int64_t cap, int32_t* out) {
  int64_t cnt = 0;
  for (int i = 0; i < n; ++i) {
    if (mask && !mask[i]) continue;
    auto nb = neighbours_of(i, n, xyz, box, mask, rc);
    for (const auto& q : nb) {
      if (cnt < cap) {
        out[2 * cnt] = i;
        out[2 * cnt + 1] = q.j;
      }
      ++cnt;
    }
  }
  return cnt;
}

int64_t oracle_neighbours_cells(int n, const double* xyz, const double* box, const uint8_t* mask,
                                double rc, int64_t cap, int32_t* out) {
  return neighbours_cells(n, xyz, box, mask, rc, cap, out);
}

// energy, forces [n,3], virial [3,3] (may be NULL), per-atom energies [n] (may be
// NULL), AEVs [n,D] and dE/dG [n,D] (may be NULL), dE/dweights (flat, may be NULL)
double oracle_energy_forces(void* mp, int n, const double* xyz, const uint8_t* sp,
                            const double* box, const uint8_t* mask, double* forces,
                            double* virial, double* atom_e, double* aev, double* dEdG,
                            double* dEdW) {
  const Model& m = *static_cast<Model*>(mp);
  if (dEdW) std::fill(dEdW, dEdW + m.flat.size(), 0.0);
  return energy_forces<double>(m, n, xyz, sp, box, mask, forces, virial, atom_e, aev, dEdG, dEdW);
}

// force-matching gradient.  v = dL/dF [n,3].  Outputs dL/dr [n,3] (= -H v) and
// dL/dweights (flat).  Forward-mode duals with tangent v through the force code.
double oracle_force_matching(void* mp, int n, const double* xyz, const uint8_t* sp,
                             const double* box, const uint8_t* mask, const double* v,
                             double* forces, double* dLdx, double* dLdw) {
  const Model& m = *static_cast<Model*>(mp);
  std::vector<Dual> x(3 * (size_t)n), F(3 * (size_t)n), dW(m.flat.size(), Dual(0.0));
  for (size_t k = 0; k < 3 * (size_t)n; ++k) x[k] = Dual(xyz[k], v[k]);
  Dual E = energy_forces<Dual>(m, n, x.data(), sp, box, mask, F.data(), nullptr, nullptr,
                               nullptr, nullptr, dW.data());
  for (size_t k = 0; k < 3 * (size_t)n; ++k) {
    if (forces) forces[k] = F[k].v;
    dLdx[k] = F[k].d;  // d/de F(r + e v) = -H v = dL/dr for L = sum (F - F_target)^2
  }
  for (size_t k = 0; k < m.flat.size(); ++k) dLdw[k] = -dW[k].d;
  return E.v;
}

// energy of a subset of centres and the forces of their terms only (the same
// per-centre work as the full sum; used to time the oracle on a bounded sample)
double oracle_energy_forces_centres(void* mp, int n, const double* xyz, const uint8_t* sp,
                                    const double* box, const uint8_t* mask, int n_centres,
                                    const int32_t* centres, double* forces) {
  const Model& m = *static_cast<Model*>(mp);
  return energy_forces<double>(m, n, xyz, sp, box, mask, forces, nullptr, nullptr, nullptr,
                               nullptr, nullptr, centres, n_centres);
}

// sampled evaluation for large systems: per-atom energies, AEV rows and forces
// on the listed atoms only (each force sums the contributions of every centre
// whose environment contains the atom).
void oracle_sample(void* mp, int n, const double* xyz, const uint8_t* sp, const double* box,
                   const uint8_t* mask, int n_sample, const int32_t* idx, double* atom_e,
                   double* forces, double* aev) {
  const Model& m = *static_cast<Model*>(mp);
  const int D = m.D();
  const double rc = std::max(m.rc_r, m.rc_a);
  std::vector<double> G(D), dG(D), dEdx(3 * (size_t)n, 0.0);
  Tape<double> tp;
  for (int t = 0; t < n_sample; ++t) {
    const int a = idx[t];
    if (atom_e) atom_e[t] = 0.0;
    for (int c = 0; c < 3; ++c) if (forces) forces[3 * t + c] = 0.0;
    if (mask && !mask[a]) {
      if (aev) for (int f = 0; f < D; ++f) aev[(size_t)t * D + f] = 0.0;
      continue;
    }
    auto nba = neighbours_of(a, n, xyz, box, mask, rc);
    std::vector<int> centres(1, a);
    for (const auto& q : nba) centres.push_back(q.j);
    double fa[3] = {0, 0, 0};
    for (int i : centres) {
      auto nb = neighbours_of(i, n, xyz, box, mask, rc);
      aev_centre(m, nb, sp, G.data());
      std::fill(dG.begin(), dG.end(), 0.0);
      double Ei = m.shift[sp[i]];
      for (int e = 0; e < m.n_ens; ++e) {
        Ei += mlp_forward(m, e, sp[i], G.data(), tp) / (double)m.n_ens;
        mlp_backward<double>(m, e, sp[i], tp, 1.0 / m.n_ens, dG.data(), nullptr);
      }
      if (i == a) {
        if (atom_e) atom_e[t] = Ei;
        if (aev) for (int f = 0; f < D; ++f) aev[(size_t)t * D + f] = G[f];
      }
      // only atom a's gradient is read, so clear the touched entries afterwards
      aev_backward_centre<double>(m, i, nb, sp, dG.data(), dEdx.data(), nullptr);
      for (int c = 0; c < 3; ++c) fa[c] -= dEdx[3 * a + c];
      dEdx[3 * i + 0] = dEdx[3 * i + 1] = dEdx[3 * i + 2] = 0.0;
      for (const auto& q : nb) dEdx[3 * q.j + 0] = dEdx[3 * q.j + 1] = dEdx[3 * q.j + 2] = 0.0;
    }
    if (forces)
      for (int c = 0; c < 3; ++c) forces[3 * t + c] = fa[c];
  }
}

}  // extern "C"
