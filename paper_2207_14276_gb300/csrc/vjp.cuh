// Buffers and launchers of the force vector-Jacobian product (double backward).
#pragma once

#include "nnp_internal.cuh"

namespace nnp {

struct VjpBufs {
  float4* v_pos;    // [n_in] dL/dF in packed order
  float4* df_pos;   // [n_in] d/de F in packed order
  float* gE_row;    // [rows] dL/dE of each row's system
  float* U;         // [rows][Dp] AEV tangent u = J v
  float* Q;         // [rows][Dp] q = H_e u
  float *H1, *D1, *Z1d, *H1d;   // [rows][E*h1]
  float *H2, *D2, *Z2d, *H2d;   // [rows][E*h2]
  float *H3, *D3, *Z3d, *H3d;   // [rows][E*h3]
  float *A1h, *A1z, *dl1, *dl1d;
  float *A2h, *A2z, *dl2, *dl2d;
  float *dl3, *dl3d;
  float* e_row;     // [E][rows]
};

struct WgradArgs {
  const float *X1, *X2;
  int ldx, x_net;
  const float *Y1, *Y2;
  int ldy, y_net;
  int n_out, n_in, n_in_real, S;
  float scale;
  float* out;
  long long per_net, layer_off;
  const int16_t* feat_of_col;   // first layer: paper index of the feature of AEV column k
};

cudaError_t vjp_set_smem(const Ws& ws);
void launch_vjp_zero(const Ws& ws, const VjpBufs& vb, int n_in, cudaStream_t st);
void launch_gather_v(const Ws& ws, const VjpBufs& vb, int n_in, cudaStream_t st);
void launch_aev_jvp(const Ws& ws, const AevConst& ac, const VjpBufs& vb, int n_in, cudaStream_t st);
void launch_aev_bwd_dual(const Ws& ws, const AevConst& ac, const VjpBufs& vb, int n_in, cudaStream_t st);
void launch_vjp_out3(const Ws& ws, const VjpBufs& vb, const float* w4, int S, int E, int h3, float alpha,
                     cudaStream_t st);
void launch_vjp_delta(const Ws& ws, int S, int width, const float* Ah, const float* Az, const float* D,
                      const float* Zd, float* dl, float* dld, float alpha, cudaStream_t st);
void launch_wgrad(const WgradArgs& a, const Ws& ws, const VjpBufs& vb, int E, cudaStream_t st);
void launch_wgrad_out(const Ws& ws, const VjpBufs& vb, int S, int E, int h3, float* out, long long per_net,
                      long long off4, cudaStream_t st);
void launch_vjp_scatter(const Ws& ws, const VjpBufs& vb, int n_in, cudaStream_t st);

}  // namespace nnp
