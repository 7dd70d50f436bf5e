// Declarations of the wall-model data kernels (k_wall.cu) and the MLP (k_mlp.cu).
#pragma once

#include <cuda_bf16.h>

#include "pnp_common.cuh"

namespace pnp {

// Index map between a fine grid and a coarse grid made of every ry-th fine
// y-face and rx x rz blocks of fine cells in x and z.
struct WallMap {
  int nx_f, nz_f, nyc_f;
  int nx_c, nz_c, nyc_c;
  int rx, ry, rz;
};

// c+, c- and Phi of a state as the wall kernels read them: the FP64 arrays, or
// (cp == nullptr) the reference profiles plus the double-float shadows of a
// mixed-precision context, c = c_ref(j) + (S + L), Phi = Phi_ref(j) + phi'.
struct IonView {
  const double *cp, *cm, *Phi;
  const float *cpS, *cpL, *cmS, *cmL, *phiS;
  const double *crefp, *crefm, *Phiref;
  __device__ __forceinline__ double cpv(int j, size_t o) const {
    return cp ? cp[o] : crefp[j] + ((double)cpS[o] + (double)cpL[o]);
  }
  __device__ __forceinline__ double cmv(int j, size_t o) const {
    return cm ? cm[o] : crefm[j] + ((double)cmS[o] + (double)cmL[o]);
  }
  __device__ __forceinline__ double phv(int j, size_t o) const { return Phi ? Phi[o] : Phiref[j] + (double)phiS[o]; }
};

template <typename T>
cudaError_t launch_restrict(const T* f, const double* dyf, const WallMap& wm, double* out, bool vfield, cudaStream_t s);
// lift: the charge-free potential of the wall model's offsets, left out of the
// features' potential (null when there are none)
template <typename TV>
cudaError_t launch_wall_features(const TV* u, const TV* w, const IonView& ions, const double* yc, const Geo& g,
                                 double V, double Uw, int ncells, const double* lift, float* X, cudaStream_t s);
template <typename TV>
cudaError_t launch_wall_labels(const TV* u, const TV* v, const TV* w, const IonView& ions, const double* ycf,
                               const double* dyf, const double* hf, const WallMap& wm, double h0c, double V,
                               double Uw, double D_ion, float* T, cudaStream_t s);
template <typename TV>
cudaError_t launch_set_slip(const float* X, int ncells, const float* Y, size_t P, double Uw, double h0b, double h0t,
                            TV* wall_u, TV* wall_w, cudaStream_t s);

// prev += w (Y - prev), Y = prev on the two wall-shear-rate columns of each row
cudaError_t launch_relax_rates(float* Y, float* prev, int rows, float w, cudaStream_t s);
// plane means of the wall-shear-rate columns, per wall, broadcast to its rows
cudaError_t launch_mean_rates(float* Y, int P, cudaStream_t s);

// wall-potential offsets B, T += gain (predicted - present first-cell potential), within +-lim;
// the present potential is the feature (without the offsets' lift) plus the lift
cudaError_t launch_edl_offsets(const float* X, int ncells, const float* Y, size_t P, double gain, double lim,
                               const double* lift, int nyc, double* B, double* T, cudaStream_t s);
// conservative transfer of ions across the first interior face of each wall
// column towards the predicted fluxes; the updated values go to the FP64
// arrays (ions.cp set) or to the shadows S, L of a mixed-precision context
template <typename TV>
cudaError_t launch_wall_flux_fix(const IonView& ions, const TV* v, const double* idy, const double* ih, const Geo& g,
                                 double Dion, const float* Y, double gain, double dt, cudaStream_t s);

// ---- MLP 40 -> 128 x 4 (erf-GELU) -> 5 ----
constexpr int kMlpLayers = 5;
constexpr int kMlpIn = 40;
constexpr int kMlpHidden = 128;
constexpr int kMlpOut = 5;

struct MlpDims {
  int in[kMlpLayers], out[kMlpLayers];
  size_t woff[kMlpLayers], boff[kMlpLayers];   // offsets in the parameter vector
  size_t nparam;
};
MlpDims mlp_dims();

// Offsets (BF16 elements) of the weight images: per layer the forward GEMM's B
// tile [Np][Kp] and the data gradient's [Kp][Np], in the shared-memory layout.
struct MlpImg {
  size_t fwd[kMlpLayers], bwd[kMlpLayers];
  size_t total;
};
MlpImg mlp_images();
cudaError_t mlp_make_images(const float* param, __nv_bfloat16* img, cudaStream_t s);

// Buffers of one MLP (all device pointers, carved by the host code).
struct MlpBufs {
  float* param;        // FP32 master weights and biases
  __nv_bfloat16* wimg; // BF16 weight images of the GEMMs (mlp_images), rebuilt from param
  float* grad;         // gradient of the loss
  float* m;            // Adam first moment
  float* v;            // Adam second moment
  float* act[kMlpLayers + 1];   // act[0] normalised input, act[l+1] output of layer l (pre-activation z)
  float* dact;         // backward scratch [B][128]
  float* dact2;        // backward scratch [B][128]
  float* partial;      // per-block partial weight gradients
  float* loss;         // [partial blocks] then the reduced loss
  float *in_shift, *in_scale, *out_shift, *out_scale;
  int* err;            // device status word (PNP_ERR_TIMEOUT from a bounded tensor-core wait)
  int skip_out = -1;   // residual output: y[skip_out] = network + x[skip_in] (none when < 0)
  int skip_in = -1;
};

// Tensor-core (tcgen05) GEMMs of the MLP (k_mlp_tc.cu).
cudaError_t mlp_fwd_layer_tc(const float* in, int K, bool act_in, const __nv_bfloat16* Wimg, const float* bias, int N,
                             int B, float* out, int* err, cudaStream_t s);
cudaError_t mlp_bwd_data_tc(const float* dz, int N, const __nv_bfloat16* WimgT, int K, int B, const float* zprev,
                            float* out, int* err, cudaStream_t s);
cudaError_t mlp_wgrad_tc(const float* dz, int N, const float* in, int K, bool act_in, int B, int rows_per_block,
                         int nblk, float* partial, int* err, cudaStream_t s);

// The whole network in one persistent kernel, outputs only (inference).
cudaError_t mlp_infer_tc(const float* X, int B, const __nv_bfloat16* wimg, const float* param,
                         const float* in_shift, const float* in_scale, const float* out_shift, const float* out_scale,
                         int skip_out, int skip_in, float* Y, int* err, cudaStream_t s);

cudaError_t mlp_sync_bf16(const MlpBufs& b, size_t nparam, cudaStream_t s);
cudaError_t mlp_forward(const MlpBufs& b, const float* X, int B, float* Y, cudaStream_t s);
cudaError_t mlp_backward(const MlpBufs& b, const float* X, const float* T, int B, int max_partial, cudaStream_t s);
cudaError_t mlp_adam(const MlpBufs& b, size_t nparam, float lr, float beta1, float beta2, float eps, int t,
                     cudaStream_t s);

}  // namespace pnp
