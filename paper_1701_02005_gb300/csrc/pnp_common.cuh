// Internal declarations shared by the libpnp CUDA translation units.
//
// Discretisation (arXiv:1701.02005, Numerical methods and Fig. 1): staggered
// second-order finite volumes, fields indexed [y][z][x].  Cell-centred fields
// (u on x-faces, w on z-faces, p, c+-, Phi at centres) have nyc planes;
// v lives on the ny = nyc + 1 y-faces, walls included (always zero).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "pnp.h"

namespace pnp {

template <typename T> struct cplx { T x, y; };

template <typename T> __host__ __device__ inline cplx<T> cadd(cplx<T> a, cplx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T> __host__ __device__ inline cplx<T> csub(cplx<T> a, cplx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T> __host__ __device__ inline cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __host__ __device__ inline cplx<T> cconj(cplx<T> a) { return {a.x, -a.y}; }

// Grid sizes and uniform x/z spacings.
struct Geo {
  int nx, nz, nyc, ny;   // ny = nyc + 1 face nodes
  int mh, mp;            // nx/2 + 1 spectral columns, padded pitch
  double dx, dz, idx, idz;
  // launch shapes chosen by the autotuner (0 = built-in default)
  int lc_rhs_bx;         // FP64 stencil: x-extent of the 128-thread blocks (16, 32, 64, 128);
                         // mixed stencil: 128 TMA rows, 64 / 32 packed-pair cp.async tiles 64 / 32
                         // cells wide, 16 one-cell tiles
  int lc_cn;             // threads per block of the wall-normal CN sweeps (mixed: 32 = shared-memory line tiles)
  int lc_spec;           // threads per block of the spectral y-solves (mixed: 16 = shared-memory tiles)
  int lc_fftz_ty;        // threads per column of the z-transform (cap)
};

// Per-y metric arrays on the device (see pnp_api.cu for definitions).
struct Metrics {
  const double* yc;    // cell centres [nyc]
  const double* idy;   // 1 / dy_j [nyc]
  const double* ih;    // 1 / h_j [ny], h = centre-to-centre distance across face j
  const double* lo_c;  // 1 / (h_j dy_j) [nyc]: coupling of cell j through face j
  const double* hi_c;  // 1 / (h_{j+1} dy_j) [nyc]: coupling through face j+1
  const double* lo_f;  // 1 / (dy_{j-1} h_j) [ny]: face j to face j-1
  const double* hi_f;  // 1 / (dy_j h_j) [ny]: face j to face j+1
  const double* wl;    // dy_{j-1} / (2 h_j) [ny]: volume weight of cell j-1 at face j
  const double* wu;    // dy_j / (2 h_j) [ny]
};

// Physical coefficients (nondimensional, Numerical methods).
struct Phys {
  double nu;   // 1/Re
  double D;    // 1/(Re Sc)
  double K;    // beta / (2 Re^2 Sc lam^2): Coulomb-force coefficient
  double q;    // 1 / (2 lam^2): Eq. (4) charge factor
  double V;    // wall potential
  double Uw;   // wall speed
};

// One RK3 substage.
struct Stage {
  double dt, gam, zet, alp;
  int af;   // approximate factorisation: x/z viscous / diffusive terms implicit (not in H)
};

// Periodic (cyclic) tridiagonal sweeps of the approximate factorisation:
// (I - s L) x = r along x or z with the constant-coefficient periodic second
// difference, by the Thomas algorithm on the corner-free system and a
// Sherman-Morrison correction: d_i = (r_i - lo d_{i-1}) m_i, y_i = d_i - c'_i
// y_{i+1}, x = y - ((y_0 + (lo / gam) y_{n-1}) fac) q.
template <typename T>
struct PeriodicFam {
  T* r;          // right-hand side / solution at the family's first plane
  int nplanes;   // planes of the family (v: the interior faces)
  const T *cp, *m, *q;   // [n] factors and the correction vector
  T lo, log, fac;        // sub-diagonal, lo / gam, 1 / (1 + q_0 + (lo / gam) q_{n-1})
};
template <typename T>
struct PeriodicArgs {
  PeriodicFam<T> f[5];
  int nfam;
};
template <typename T>
cudaError_t launch_periodic(const PeriodicArgs<T>& a, const Geo& g, bool zdir, cudaStream_t s);

// The same x and z sweeps as truncated circulant convolutions, both directions
// in one pass (launch_periodic_conv): the inverse of each constant-coefficient
// cyclic system is x_i = sum_k g_k r_(i-k), g symmetric and decaying
// geometrically; taps g_0 .. g_K past which the dropped tail is below the
// arithmetic's rounding.
constexpr int kConvMaxK = 8;
template <typename T>
struct ConvFam {
  T* r;          // right-hand side / solution at the family's first plane
  int nplanes;   // planes of the family (v: the interior faces)
  int kx;        // x taps beyond the centre (<= kConvMaxK)
  T gx[kConvMaxK + 1], gz[kConvMaxK + 1];   // g_0 .. g_K along x and z (z: zero past the family's K)
};
template <typename T>
struct ConvArgs {
  ConvFam<T> f[5];
  int nfam;
  int kz;   // z taps beyond the centre of the launch: 1, 2, 4 or 8 (the families' largest, rounded up)
};
template <typename T>
cudaError_t launch_periodic_conv(const ConvArgs<T>& a, const Geo& g, cudaStream_t s);

template <typename TV>
struct Fields {
  TV *u, *v, *w, *p;
  TV *Hu, *Hv, *Hw;
  TV *ru, *rv, *rw;
  double *cp, *cm, *Phi;
  double *Hcp, *Hcm;
  double *rcp, *rcm;
  // optional per-column wall velocities [2][nz][nx] (bottom, top), lab frame;
  // nullptr = the uniform wall speeds -Uw / +Uw for u and 0 for w
  const TV *wall_u, *wall_w;
};

// Crank-Nicolson factor rows of one substage for the y-implicit solves:
// forward elimination d_j = (r_j - a_j d_{j-1}) m_j, back substitution
// x_j = d_j - c_j x_{j+1}.  a, c, m are arrays of the line length.
struct CNRows {
  const double *a, *c, *m;
};

// Rows (a, b, c) of the wall-normal second difference of a cell-centred
// quantity, used by the spectral Thomas solves.
struct YRows {
  const double *a, *b, *c;
};

__host__ __device__ inline size_t cidx(int j, int k, int i, int nz, int nx) {
  return ((size_t)j * nz + k) * nx + i;
}

// ---- launchers (host functions; all asynchronous on stream) ----
template <typename TV>
cudaError_t launch_rhs(const Fields<TV>& f, const Geo& g, const Metrics& m, const Phys& ph,
                       const Stage& st, cudaStream_t s);

template <typename TV>
cudaError_t launch_cn_solves(const Fields<TV>& f, const Geo& g, const CNRows& vel, const CNRows& face,
                             const CNRows& ion, cudaStream_t s);

// Poisson pipeline pieces.  Spectral buffer holds (nyc, nz, mp) complex T.
// ChargeShadowDF: the fluctuating charge from the double-float ion state
// (high parts sa, sb and low parts la, lb), formed in the transform's precision.
enum class PoissonSrc { Divergence, Charge, ChargeShadow, ChargeShadowDF, Plain };
enum class PoissonDst { Plain, Potential, PotentialShadow };

template <typename T, typename TV>
cudaError_t launch_fft_x_fwd(PoissonSrc src, const TV* u, const TV* v, const TV* w, const double* cp,
                             const double* cm, const T* plain, double scale, const Geo& g,
                             const Metrics& m, cplx<T>* spec, const cplx<T>* tw_half,
                             const cplx<T>* tw_post, cudaStream_t s, const float* sa = nullptr,
                             const float* sb = nullptr, const T* idyT = nullptr, const float* la = nullptr,
                             const float* lb = nullptr);

template <typename T>
cudaError_t launch_fft_z(cplx<T>* spec, const cplx<T>* tw_z, const Geo& g, bool inverse, cudaStream_t s);

// Elimination factors of the spectral y-solves (grid-only, computed once).
cudaError_t launch_spec_factors(double* cpr, double* inv, const double* kx2, const double* kz2, const YRows& rows,
                                const Geo& g, bool neumann, cudaStream_t s);

// Double-float copies of the spectral elimination factors (mixed path).
struct SpecDF {
  const float2 *cpr, *inv;   // per spectral point, same layout as the FP64 factors
  const float2* a;           // sub-diagonal of the y-operator per plane
};
cudaError_t launch_spec_thomas_df(cplx<float>* spec, void* dscr, const SpecDF& f, const double* cpr,
                                  const double* inv, const YRows& rows, const Geo& g, double scale, bool neumann,
                                  cudaStream_t s, const double* mean_rhs = nullptr,
                                  const double* mean_shift = nullptr, double* mean_out = nullptr);
cudaError_t launch_to_df(const double* x, float2* out, size_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_spec_thomas(cplx<T>* spec, cplx<double>* dscr, const double* cpr, const double* inv,
                               const YRows& rows, const Geo& g, double scale, bool neumann, cudaStream_t s,
                               const double* mean_rhs = nullptr, const double* mean_shift = nullptr,
                               double* mean_out = nullptr);

// Potential / PotentialShadow: out = V yc_j (Potential) or plane_add[j]
// (PotentialShadow) + the transform + cell_add[c] (optional, per cell).
template <typename T, typename TO>
cudaError_t launch_fft_x_inv(PoissonDst dst, const cplx<T>* spec, const Geo& g, const Metrics& m,
                             const cplx<T>* tw_half, const cplx<T>* tw_post, double V, TO* out,
                             cudaStream_t s, const double* plane_add = nullptr, const TO* cell_add = nullptr);

// Wall potentials that vary along the walls: the source -(d_xx + d_zz) Phi_0'
// of the zero-mean part of the linear lift Phi_0' = (1 - y)/2 (B - Bm) +
// (1 + y)/2 (T - Tm) (B, T the [nz][nx] wall values, Bm, Tm their means),
// and, after the Dirichlet solve, lift64 += Phi_0' + off and lift32 = the
// FP32 value without off.
cudaError_t launch_wall_lift_source(double* src, const double* B, const double* T, double Bm, double Tm,
                                    const double* yc, const Geo& g, cudaStream_t s);
cudaError_t launch_wall_lift_finish(double* lift64, float* lift32, const double* B, const double* T, double Bm,
                                    double Tm, double off, const double* yc, const Geo& g, cudaStream_t s);

template <typename T>
cudaError_t launch_project(T* u, T* v, T* w, T* p, const T* phip, double scale, bool update_p, const Geo& g,
                           const T* ih, cudaStream_t s);

// Initial condition, diagnostics, conversions.
template <typename TV>
cudaError_t launch_init_fields(const Fields<TV>& f, const Geo& g, const Metrics& m, const Phys& ph,
                               int ic_kind, double cb, double kappa, uint64_t seed, double amp,
                               const double* yf, cudaStream_t s);

// Stability limits checked by the diagnostics pass (device status word):
// dt = the last step's size (<= 0: no CFL check), cfl_max = bound on
// dt (|u|/dx + |v|/dy + |w|/dz), dphi_max = bound on the potential step
// between neighbouring cells (2: the positivity limit of the discrete
// Boltzmann ratio (2 - dPhi) / (2 + dPhi) of the arithmetic face means).
struct DiagLimits {
  double dt, cfl_max, dphi_max;
};
constexpr int kDiagOutSlots = 14;   // doubles written by the final diagnostics reduction

template <typename TV>
cudaError_t launch_diagnostics(const Fields<TV>& f, const Geo& g, const Metrics& m, const Phys& ph,
                               double* partial, int npartial, double* out, int* status, const DiagLimits& lim,
                               cudaStream_t s);

template <typename TA, typename TB>
cudaError_t launch_convert(const TA* a, TB* b, size_t n, cudaStream_t s);

template <typename TQ>
cudaError_t launch_mean_profile(const TQ* q, int nplanes, int plane, double* out, cudaStream_t s);

cudaError_t launch_fp64_probe(double* out, int iters, int blocks, cudaStream_t s);

}  // namespace pnp
