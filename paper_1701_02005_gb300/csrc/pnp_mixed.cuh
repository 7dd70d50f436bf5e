// Declarations of the mixed-precision path (see k_mixed.cu for the policy).
#pragma once

#include <cuda.h>

#include "pnp_common.cuh"

namespace pnp {

// FP32 copies of the per-y metric arrays (same meaning as Metrics).
struct MetricsF {
  const float *idy, *ih, *lo_c, *hi_c, *lo_f, *hi_f, *wl, *wu;
};

// FP32 copies of the scalar coefficients of one substage (converted once on
// the host: per-thread FP64->FP32 conversions run on the FP64 pipe).
struct CoefF {
  float idx, idz, nu, D, K, Uw;
  float dt, gam, zet, alp;
  // products used per cell, formed once in FP32 on the host
  float idx2, idz2, Kx, Kz, Dx, Dz, anu, aD;
  // 0: the explicit terms H of this substage are not stored (the low-storage
  // RK3's last substage: the next step's first substage has zeta = 0 and never
  // reads them); the previous H is read only when zet != 0
  int keep_h;
  // approximate factorisation (0 = off): x/z viscous / diffusive terms leave H and
  // join the implicit side: nuH = 0, anuxz = alp nu (momentum r += anuxz lap_xz);
  // ions H -= D lap_xz c', r += dt zet D lap_xz c'
  int af;
  float nuH, anuxz, zD;
};

// FP32 elimination factors of the velocity Crank-Nicolson matrices.
struct CNRowsF {
  const float *a, *c, *m;
};

// FP32 fluctuation shadows (relative to the reference profiles).
struct Shadows {
  float *cp, *cm;    // c+' , c-' (high parts of the df ion fluctuations)
  float *phi;        // phi' = Phi - Phi_ref
  float *Hcp, *Hcm;  // explicit ion terms minus their reference part
  float *cpL, *cmL;  // low parts: c = c_ref + cp + cpL exactly to the df resolution
};

// Per-plane reference data.  FP32 arrays feed the FP32 stencils; FP64 arrays
// hold the exact reference and the folded reference-reference terms.
struct MixedRefs {
  const float *cref_p, *cref_m;   // c_ref per cell plane [nyc]
  const float *crf_p, *crf_m;     // 0.5 (c_ref_{j-1} + c_ref_j) per interior y-face [ny]
  const float* rho_ref;           // c+_ref - c-_ref [nyc]
  const float* rhorf;             // face mean of rho_ref [ny]
  const float* dPref;             // Phi_ref_j - Phi_ref_{j-1} per interior face [ny]
  const float* Fvref;             // -K rhorf dPref / h: reference Coulomb force on v [ny]
  const double *Rref_p, *Rref_m;  // [3][nyc]: reference increments (I - s_l L_y)^-1 dt alp_l (H_ref + D L_y c_ref)
  const double *cref64_p, *cref64_m, *Phiref64;   // exact references [nyc]
  const double* mean_rhs;         // -q rho_ref [nyc]: FP64 (0,0) mode source of Eq. (4)
  const double* mean_shift;       // V y_c - Phi_ref [nyc]
  double* delta;                  // [nyc] written each solve: V y_c + phi_mean - Phi_ref
  const float2 *dC_p, *dC_m;      // [3][nyc]: Rref_p, Rref_m as df pairs (the ion update adds them)
};

// TMA descriptors of the stencil inputs and old H arrays of one context
// (3-D {nx, nz, planes} float tensors, one x-row per copy).
struct RhsMaps {
  CUtensorMap t[7];   // u, w, v, p, phi', c+', c-'
  CUtensorMap h[5];   // Hu, Hw, Hv, Hc+', Hc-'
};

bool rhs_tma_eligible(const Geo& g);
// One bounded mbarrier wait that cannot complete (failure-path self-test).
// Diagnostics partial sums from the FP32 fields and the df ion state (no FP64
// copy); wgt[j] = dy_j and wgt[2 ny + j] = 1/dy_j (j < nyc), wgt[ny + j] = h_j,
// as df pairs; dPref[j] the reference potential step across interior face j.
// The reference parts of the ion numbers and of the explicit ion terms are not
// included.
cudaError_t launch_diagnostics_mixed(const Fields<float>& f, const Shadows& sh, const float* cref_p,
                                     const float* cref_m, const float* dPref, const float2* wgt, const Geo& g,
                                     double* partial, int npartial, double* out, int* status,
                                     const DiagLimits& lim, cudaStream_t s);
cudaError_t launch_wait_selftest(int* err, double limit_s, cudaStream_t s);
cudaError_t build_rhs_maps(RhsMaps* m, const Fields<float>& f, const Shadows& sh, const Geo& g);
// The CN forward elimination fused into the stencil (on != 0): the substage's
// FP32 factor rows of the three families (cells u, w; v faces; ions) and the
// y-chunk length the stencil marches, which the back substitution must know.
struct CnFuse {
  CNRowsF cell, face, ion;
  int jc;
  int on;
};
// Planes per y-chunk of the stencil launch_mixed_rhs takes on this grid and
// launch shape (tma_maps: the context has the TMA tensor maps).
int mixed_rhs_chunk(const Geo& g, bool tma_maps);
// maps == nullptr selects the cp.async tile kernel; err receives PNP_ERR_TIMEOUT
// if a TMA copy does not complete within the kernel's wait limit.  fuse (optional):
// store d~ (chunk-local forward elimination) instead of the CN right-hand sides.
cudaError_t launch_mixed_rhs(const Fields<float>& f, const Shadows& sh, const MixedRefs& R, const Geo& g,
                             const MetricsF& m, const CoefF& cf, const RhsMaps* maps, int* err, cudaStream_t s,
                             const CnFuse* fuse = nullptr);
// Back substitution of the wall-normal CN solves after the fused stencil: per
// line, the chunk-boundary values of the forward elimination from the chunks'
// d~ and the products G (tables [row] per family: cells, faces, ions), then
// x_j = d_j - c_j x_{j+1} from the top with d_j = d~_j + G_j d_{s-1}.
struct CnFusedG {
  const float *cell, *face, *ion;
};
cudaError_t launch_mixed_cn_fused(const Fields<float>& f, const Shadows& sh, const MixedRefs& R, const Geo& g,
                                  const CNRowsF& cell, const CNRowsF& face, const CNRowsF& ion, const CnFusedG& G,
                                  int jc, int l, unsigned parts, cudaStream_t s);
constexpr int kFusedMaxChunks = 32;
// Wall-normal CN solves of substage l: the ion families and / or the velocity families.
constexpr unsigned kCnIons = 1, kCnVelocity = 2;
cudaError_t launch_mixed_cn(const Fields<float>& f, const Shadows& sh, const MixedRefs& R, const Geo& g,
                            const CNRowsF& cell, const CNRowsF& face, const CNRowsF& ion, int l, unsigned parts,
                            cudaStream_t s);
// Sources of a statistics sample (FP64 path: the FP64 arrays; mixed: FP32
// velocities, the double-float ion state and phi' about the FP64 references).
struct StatSrc {
  const void *u, *v, *w;
  bool vel_f32, mixed;
  const double *cp, *cm, *Phi;
  const float *cpS, *cpL, *cmS, *cmL, *phiS;
  const double *cref_p, *cref_m, *phi_ref;
};
cudaError_t launch_stats_sample(const StatSrc& src, const Geo& g, double* acc, cudaStream_t s);

// FP64 scratch of the FP64-arithmetic CN solves: forward values per line
// (du, dw, dcp, dcm: nyc planes; dv: ny planes).
struct CnScratch64 {
  double *du, *dv, *dw, *dcp, *dcm;
};
cudaError_t launch_mixed_cn_fp64(const Fields<float>& f, const Shadows& sh, const MixedRefs& R, const Geo& g,
                                 const CNRows& cell, const CNRows& face, const CNRows& ion, int l, unsigned parts,
                                 const CnScratch64& scr, cudaStream_t s);
cudaError_t launch_plane_means3(const double* a, const double* b, const double* c, int nplanes, size_t P,
                                double* oa, double* ob, double* oc, cudaStream_t s);
cudaError_t launch_make_shadows(const double* cp, const double* cm, const double* Phi, const double* Hcp,
                                const double* Hcm, const Shadows& sh, const MixedRefs& R, const double* Href_p,
                                const double* Href_m, size_t P, size_t n, cudaStream_t s);
cudaError_t launch_from_shadow_df(const float* S, const float* L, const double* ref, double* out, size_t P, size_t n,
                                  cudaStream_t s);
cudaError_t launch_from_shadow(const float* sh, const double* ref, double* out, size_t P, size_t n, cudaStream_t s);


}  // namespace pnp
