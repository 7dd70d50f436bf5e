// Mixed-precision kernels of the fractional step (arXiv:1701.02005, Eqs. (1)-(4),
// Numerical methods; staggering of Fig. 1).
//
// Precision policy.  Ion concentrations c+- stay FP64 in memory and every
// wall-normal solve (ion Crank-Nicolson, both Poisson y-solves, the (0,0)
// mean mode of the potential) runs in FP64.  The stencils run in FP32 on
// shadows relative to FP64 reference profiles of y:
//     c = c_ref(y) + c',   Phi = Phi_ref(y) + phi',
// c_ref, Phi_ref being plane means taken when the state is loaded.  Every
// product of two reference quantities (the 1-D double-layer migration flux,
// its divergence, the implicit diffusion of c_ref and the osmotic Coulomb
// force on v) is a per-plane FP64 constant folded in exactly; only terms that
// contain a fluctuation are rounded to FP32, so the near-cancellation of
// diffusion and migration inside the Debye layer happens in FP64.
// Velocities, pressure and the momentum stencils are FP32; the velocity
// Crank-Nicolson matrix is I - s L_y with s L_y = O(1) (well conditioned) and
// runs in FP32.
#include "pnp_common.cuh"
#include "pnp_mixed.cuh"

namespace pnp {

__device__ __forceinline__ float Lf(const float* p, size_t i) { return __ldg(p + i); }

// ---------------------------------------------------------------------------
// Right-hand sides in FP32, one pass per cell: momentum (u, w on every cell;
// v on faces j >= 1), then both ions, reusing the loaded velocities and
// shadows.  For the ions the CN right-hand side is split as r_c = Rref(j) + r',
// Rref the per-plane FP64 reference part (solved once per substage on the
// host, see k_cn_ion_mixed) and r' = dt [gam H' + zet H'_old + alp D L_y c']
// stored in FP32.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_rhs_mixed(Fields<float> f, float* __restrict__ rcp, float* __restrict__ rcm,
                                                   Shadows sh, MixedRefs R, Geo g, MetricsF mt, CoefF cf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.z;
  if (i >= g.nx || k >= g.nz) return;
  const int nx = g.nx, nz = g.nz, nyc = g.nyc;
  const int im = i ? i - 1 : nx - 1, ip = (i + 1 == nx) ? 0 : i + 1;
  const int km = k ? k - 1 : nz - 1, kp = (k + 1 == nz) ? 0 : k + 1;
  const bool has_dn = j > 0, has_up = j < nyc - 1;
  const float idx = cf.idx, idz = cf.idz;
  const float idx2 = idx * idx, idz2 = idz * idz;
  const size_t c0 = cidx(j, k, i, nz, nx);
  const size_t cxm = cidx(j, k, im, nz, nx), cxp = cidx(j, k, ip, nz, nx);
  const size_t czm = cidx(j, km, i, nz, nx), czp = cidx(j, kp, i, nz, nx);
  const size_t P = (size_t)nz * nx;
  const float idyj = mt.idy[j];
  const float nu = cf.nu, K = cf.K, Uw = cf.Uw;
  const float dt = cf.dt, gam = cf.gam, zet = cf.zet, alp = cf.alp;

  const float u0 = Lf(f.u, c0), uxm = Lf(f.u, cxm), uxp = Lf(f.u, cxp), uzm = Lf(f.u, czm), uzp = Lf(f.u, czp);
  const float uym = has_dn ? Lf(f.u, c0 - P) : 0.f, uyp = has_up ? Lf(f.u, c0 + P) : 0.f;
  const float w0 = Lf(f.w, c0), wxm = Lf(f.w, cxm), wxp = Lf(f.w, cxp), wzm = Lf(f.w, czm), wzp = Lf(f.w, czp);
  const float wym = has_dn ? Lf(f.w, c0 - P) : 0.f, wyp = has_up ? Lf(f.w, c0 + P) : 0.f;
  const float vb = Lf(f.v, c0), vt = Lf(f.v, c0 + P);
  const float p0 = Lf(f.p, c0);
  const float ph0 = Lf(sh.phi, c0), phxm = Lf(sh.phi, cxm), phxp = Lf(sh.phi, cxp);
  const float phzm = Lf(sh.phi, czm), phzp = Lf(sh.phi, czp);
  const float phym = has_dn ? Lf(sh.phi, c0 - P) : 0.f, phyp = has_up ? Lf(sh.phi, c0 + P) : 0.f;
  const float cp0 = Lf(sh.cp, c0), cm0 = Lf(sh.cm, c0);
  const float rho0 = cp0 - cm0;   // rho' at the centre
  const float rref = R.rho_ref[j];

  // u at (x-face i, y-centre j, z-centre k)
  {
    const float ubp = 0.5f * (u0 + uxp), ubm = 0.5f * (uxm + u0);
    const float ax = (ubp * ubp - ubm * ubm) * idx;
    const float vft = 0.5f * (Lf(f.v, cidx(j + 1, k, im, nz, nx)) + vt);
    const float vfb = 0.5f * (Lf(f.v, cxm) + vb);
    const float uft = has_up ? 0.5f * (u0 + uyp) : 0.f;
    const float ufb = has_dn ? 0.5f * (uym + u0) : 0.f;
    const float ay = (vft * uft - vfb * ufb) * idyj;
    const float wfk = 0.5f * (wxm + w0);
    const float wfkp = 0.5f * (Lf(f.w, cidx(j, kp, im, nz, nx)) + wzp);
    const float az = (wfkp * 0.5f * (u0 + uzp) - wfk * 0.5f * (uzm + u0)) * idz;
    const float lap = (uxp - 2.f * u0 + uxm) * idx2 + (uzp - 2.f * u0 + uzm) * idz2;
    const float rhom = Lf(sh.cp, cxm) - Lf(sh.cm, cxm);
    const float fu = -K * (rref + 0.5f * (rhom + rho0)) * (ph0 - phxm) * idx;
    const float H = -(ax + ay + az) + nu * lap + fu;
    const float ub = f.wall_u ? f.wall_u[(size_t)k * nx + i] : -Uw;
    const float ut = f.wall_u ? f.wall_u[P + (size_t)k * nx + i] : Uw;
    const float Ly = mt.lo_c[j] * ((has_dn ? uym : ub) - u0) + mt.hi_c[j] * ((has_up ? uyp : ut) - u0);
    const float gp = (p0 - Lf(f.p, cxm)) * idx;
    const float Ho = f.Hu[c0];
    f.ru[c0] = dt * (gam * H + zet * Ho - alp * gp + alp * nu * Ly);
    f.Hu[c0] = H;
  }
  // w at (x-centre i, y-centre j, z-face k)
  {
    const float wbp = 0.5f * (w0 + wzp), wbm = 0.5f * (wzm + w0);
    const float az = (wbp * wbp - wbm * wbm) * idz;
    const float vft = 0.5f * (Lf(f.v, cidx(j + 1, km, i, nz, nx)) + vt);
    const float vfb = 0.5f * (Lf(f.v, czm) + vb);
    const float wft = has_up ? 0.5f * (w0 + wyp) : 0.f;
    const float wfb = has_dn ? 0.5f * (wym + w0) : 0.f;
    const float ay = (vft * wft - vfb * wfb) * idyj;
    const float ufi = 0.5f * (uzm + u0);
    const float ufip = 0.5f * (Lf(f.u, cidx(j, km, ip, nz, nx)) + uxp);
    const float ax = (ufip * 0.5f * (w0 + wxp) - ufi * 0.5f * (wxm + w0)) * idx;
    const float lap = (wxp - 2.f * w0 + wxm) * idx2 + (wzp - 2.f * w0 + wzm) * idz2;
    const float rhom = Lf(sh.cp, czm) - Lf(sh.cm, czm);
    const float fw = -K * (rref + 0.5f * (rhom + rho0)) * (ph0 - phzm) * idz;
    const float H = -(ax + ay + az) + nu * lap + fw;
    const float wb = f.wall_w ? f.wall_w[(size_t)k * nx + i] : 0.f;
    const float wt = f.wall_w ? f.wall_w[P + (size_t)k * nx + i] : 0.f;
    const float Ly = mt.lo_c[j] * ((has_dn ? wym : wb) - w0) + mt.hi_c[j] * ((has_up ? wyp : wt) - w0);
    const float gp = (p0 - Lf(f.p, czm)) * idz;
    const float Ho = f.Hw[c0];
    f.rw[c0] = dt * (gam * H + zet * Ho - alp * gp + alp * nu * Ly);
    f.Hw[c0] = H;
  }
  // v at (x-centre i, y-face j, z-centre k), 1 <= j <= nyc-1
  if (has_dn) {
    const float wl = mt.wl[j], wu = mt.wu[j], ihj = mt.ih[j];
    const size_t d0 = c0 - P;
    const float v0 = vb;
    const float vxm = Lf(f.v, cxm), vxp = Lf(f.v, cxp), vzm = Lf(f.v, czm), vzp = Lf(f.v, czp);
    const float vym = Lf(f.v, c0 - P), vyp = vt;
    const float Ui = wl * Lf(f.u, d0) + wu * u0;
    const float Uip = wl * Lf(f.u, cidx(j - 1, k, ip, nz, nx)) + wu * uxp;
    const float ax = (Uip * 0.5f * (v0 + vxp) - Ui * 0.5f * (vxm + v0)) * idx;
    const float vbu = 0.5f * (v0 + vyp), vbd = 0.5f * (vym + v0);
    const float ay = (vbu * vbu - vbd * vbd) * ihj;
    const float Wk = wl * Lf(f.w, d0) + wu * w0;
    const float Wkp = wl * Lf(f.w, cidx(j - 1, kp, i, nz, nx)) + wu * wzp;
    const float az = (Wkp * 0.5f * (v0 + vzp) - Wk * 0.5f * (vzm + v0)) * idz;
    const float lap = (vxp - 2.f * v0 + vxm) * idx2 + (vzp - 2.f * v0 + vzm) * idz2;
    // Coulomb force: reference-reference part is the FP64 constant Fvref
    const float rhod = Lf(sh.cp, d0) - Lf(sh.cm, d0);
    const float rpf = 0.5f * (rhod + rho0);                 // rho' on the face
    const float dphi = ph0 - phym;                          // phi' difference
    const float fv = R.Fvref[j] - K * ihj * (R.rhorf[j] * dphi + rpf * (R.dPref[j] + dphi));
    const float H = -(ax + ay + az) + nu * lap + fv;
    const float Ly = mt.lo_f[j] * (vym - v0) + mt.hi_f[j] * (vyp - v0);
    const float gp = (p0 - Lf(f.p, d0)) * ihj;
    const float Ho = f.Hv[c0];
    f.rv[c0] = dt * (gam * H + zet * Ho - alp * gp + alp * nu * Ly);
    f.Hv[c0] = H;
  }

  // ---- ions: FP32 fluctuation fluxes (the reference-reference part is in Rref) ----
  {
    const float D = cf.D;
    const float ihj = mt.ih[j], ihjp = mt.ih[j + 1];
    const float lo = mt.lo_c[j], hi = mt.hi_c[j];
#pragma unroll
    for (int ion = 0; ion < 2; ++ion) {
      const float* c = ion == 0 ? sh.cp : sh.cm;
      const float s = ion == 0 ? 1.f : -1.f;
      const float cr = ion == 0 ? R.cref_p[j] : R.cref_m[j];
      const float* crf = ion == 0 ? R.crf_p : R.crf_m;
      const float cc = ion == 0 ? cp0 : cm0;
      const float cxm_ = Lf(c, cxm), cxp_ = Lf(c, cxp), czm_ = Lf(c, czm), czp_ = Lf(c, czp);
      const float cym_ = has_dn ? Lf(c, c0 - P) : 0.f, cyp_ = has_up ? Lf(c, c0 + P) : 0.f;
      // x and z faces: the reference is uniform in the plane, so only c', phi' differences appear
      float ca = cr + 0.5f * (cxm_ + cc), cb = cr + 0.5f * (cc + cxp_);
      const float Fx_i = u0 * ca - D * (cc - cxm_) * idx - s * D * ca * (ph0 - phxm) * idx;
      const float Fx_ip = uxp * cb - D * (cxp_ - cc) * idx - s * D * cb * (phxp - ph0) * idx;
      ca = cr + 0.5f * (czm_ + cc);
      cb = cr + 0.5f * (cc + czp_);
      const float Fz_k = w0 * ca - D * (cc - czm_) * idz - s * D * ca * (ph0 - phzm) * idz;
      const float Fz_kp = wzp * cb - D * (czp_ - cc) * idz - s * D * cb * (phzp - ph0) * idz;
      // y faces: advection + migration
      float Fy_j = 0.f, Fy_jp = 0.f;
      if (has_dn) {
        const float cpf = 0.5f * (cym_ + cc), dph = ph0 - phym;
        Fy_j = vb * (crf[j] + cpf) - s * D * (crf[j] * dph + cpf * (R.dPref[j] + dph)) * ihj;
      }
      if (has_up) {
        const float cpf = 0.5f * (cc + cyp_), dph = phyp - ph0;
        Fy_jp = vt * (crf[j + 1] + cpf) - s * D * (crf[j + 1] * dph + cpf * (R.dPref[j + 1] + dph)) * ihjp;
      }
      const float H = -((Fx_ip - Fx_i) * idx + (Fy_jp - Fy_j) * idyj + (Fz_kp - Fz_k) * idz);
      const float Ly = (has_dn ? lo * (cym_ - cc) : 0.f) + (has_up ? hi * (cyp_ - cc) : 0.f);
      float* Hc = ion == 0 ? sh.Hcp : sh.Hcm;
      float* rc = ion == 0 ? rcp : rcm;
      const float Ho = Hc[c0];
      rc[c0] = dt * (gam * H + zet * Ho + alp * D * Ly);
      Hc[c0] = H;
    }
  }
}

// ---------------------------------------------------------------------------
// Ion Crank-Nicolson solve.  (I - s L_y) dc = Rref + r' is linear, so
// dc = dC_ref + (I - s L_y)^-1 r' with dC_ref the FP64 reference increment of
// the substage (a 1-D solve done on the host).  The fluctuation part runs in
// FP32; only the state update c <- c + dC_ref + x' (and the shadow
// c' = c - c_ref) is FP64.
// ---------------------------------------------------------------------------
__global__ void k_cn_ion_mixed(double* __restrict__ cp, float* __restrict__ rcp, float* __restrict__ sp,
                               double* __restrict__ cm, float* __restrict__ rcm, float* __restrict__ sm,
                               CNRowsF rows, const double* __restrict__ dCp, const double* __restrict__ dCm,
                               MixedRefs R, int n, size_t P) {
  constexpr int CH = 8;   // planes loaded ahead per sweep step
  const size_t line = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= P) return;
  const bool plus = blockIdx.y == 0;
  double* q = plus ? cp : cm;
  float* r = plus ? rcp : rcm;
  float* s = plus ? sp : sm;
  const double* cref = plus ? R.cref64_p : R.cref64_m;
  const double* dC = plus ? dCp : dCm;
  float d = 0.f;
  for (int jb = 0; jb < n; jb += CH) {
    float rr[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u)
      if (jb + u < n) rr[u] = r[(size_t)(jb + u) * P + line];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int j = jb + u;
      if (j < n) {
        d = (rr[u] - rows.a[j] * d) * rows.m[j];
        r[(size_t)j * P + line] = d;
      }
    }
  }
  float x = 0.f;
  for (int jb = n - 1; jb >= 0; jb -= CH) {
    float dd[CH];
    double qq[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u)
      if (jb - u >= 0) {
        const size_t o = (size_t)(jb - u) * P + line;
        dd[u] = r[o];
        qq[u] = q[o];
      }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int j = jb - u;
      if (j >= 0) {
        const size_t o = (size_t)j * P + line;
        x = dd[u] - rows.c[j] * x;
        const double cn = (qq[u] + dC[j]) + (double)x;
        q[o] = cn;
        s[o] = (float)(cn - cref[j]);
      }
    }
  }
}

// FP32 velocity Crank-Nicolson solves (u, w: nyc cells; v: interior faces).
__global__ void k_cn_vel_f32(float* __restrict__ u, float* __restrict__ ru, float* __restrict__ v,
                             float* __restrict__ rv, float* __restrict__ w, float* __restrict__ rw,
                             CNRowsF cell, CNRowsF face, int nyc, size_t P) {
  constexpr int CH = 8;
  const size_t line = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= P) return;
  float* q;
  float* r;
  CNRowsF rw_;
  int n, j0;
  if (blockIdx.y == 0) { q = u; r = ru; rw_ = cell; n = nyc; j0 = 0; }
  else if (blockIdx.y == 1) { q = v; r = rv; rw_ = face; n = nyc - 1; j0 = 1; }
  else { q = w; r = rw; rw_ = cell; n = nyc; j0 = 0; }
  float* rl = r + (size_t)j0 * P + line;
  float* ql = q + (size_t)j0 * P + line;
  float d = 0.f;
  for (int jb = 0; jb < n; jb += CH) {
    float rr[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (jb + k < n) rr[k] = rl[(size_t)(jb + k) * P];
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      const int j = jb + k;
      if (j < n) {
        d = (rr[k] - rw_.a[j] * d) * rw_.m[j];
        rl[(size_t)j * P] = d;
      }
    }
  }
  float x = 0.f;
  for (int jb = n - 1; jb >= 0; jb -= CH) {
    float dd[CH], qq[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (jb - k >= 0) {
        dd[k] = rl[(size_t)(jb - k) * P];
        qq[k] = ql[(size_t)(jb - k) * P];
      }
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      const int j = jb - k;
      if (j >= 0) {
        x = dd[k] - rw_.c[j] * x;
        ql[(size_t)j * P] = qq[k] + x;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Reference profiles: deterministic FP64 plane means (one block per plane).
// ---------------------------------------------------------------------------
__global__ void k_plane_means3(const double* __restrict__ a, const double* __restrict__ b,
                               const double* __restrict__ c, size_t P, double* out_a, double* out_b,
                               double* out_c) {
  __shared__ double sh[3][256];
  const int j = blockIdx.x;
  double sa = 0.0, sb = 0.0, sc = 0.0;
  for (size_t t = threadIdx.x; t < P; t += blockDim.x) {
    const size_t o = (size_t)j * P + t;
    sa += a[o];
    sb += b[o];
    sc += c[o];
  }
  sh[0][threadIdx.x] = sa;
  sh[1][threadIdx.x] = sb;
  sh[2][threadIdx.x] = sc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + st];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + st];
      sh[2][threadIdx.x] += sh[2][threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out_a[j] = sh[0][0] / (double)P;
    out_b[j] = sh[1][0] / (double)P;
    out_c[j] = sh[2][0] / (double)P;
  }
}

// Shadows from full FP64 fields: c' = c - c_ref, phi' = Phi - Phi_ref, H' = H - H_ref.
__global__ void k_make_shadows(const double* __restrict__ cp, const double* __restrict__ cm,
                               const double* __restrict__ Phi, const double* __restrict__ Hcp,
                               const double* __restrict__ Hcm, Shadows sh, MixedRefs R, const double* Href_p,
                               const double* Href_m, size_t P, size_t n) {
  const size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const int j = (int)(o / P);
  sh.cp[o] = (float)(cp[o] - R.cref64_p[j]);
  sh.cm[o] = (float)(cm[o] - R.cref64_m[j]);
  sh.phi[o] = (float)(Phi[o] - R.Phiref64[j]);
  sh.Hcp[o] = (float)(Hcp[o] - Href_p[j]);
  sh.Hcm[o] = (float)(Hcm[o] - Href_m[j]);
}

// Full FP64 fields from shadows: X = X_ref(j) + (double) X'.
__global__ void k_from_shadow(const float* __restrict__ s, const double* __restrict__ ref, double* __restrict__ out,
                              size_t P, size_t n) {
  const size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  out[o] = ref[o / P] + (double)s[o];
}

// ---------------------------------------------------------------------------
cudaError_t launch_mixed_rhs(const Fields<float>& f, const Shadows& sh, const MixedRefs& R, const Geo& g,
                             const MetricsF& m, const CoefF& cf, int l, cudaStream_t s) {
  const int bx = g.lc_rhs_bx ? g.lc_rhs_bx : 32, by = 128 / bx;
  dim3 blk(bx, by, 1);
  dim3 grd((g.nx + bx - 1) / bx, (g.nz + by - 1) / by, g.nyc);
  (void)l;
  k_rhs_mixed<<<grd, blk, 0, s>>>(f, reinterpret_cast<float*>(f.rcp), reinterpret_cast<float*>(f.rcm), sh, R, g, m, cf);
  return cudaGetLastError();
}

cudaError_t launch_mixed_cn(const Fields<float>& f, const Shadows& sh, const MixedRefs& R, const Geo& g,
                            const CNRowsF& cell, const CNRowsF& face, const CNRowsF& ion, int l, cudaStream_t s) {
  const size_t P = (size_t)g.nz * g.nx;
  const int T = g.lc_cn ? g.lc_cn : 128;
  dim3 grd((unsigned)((P + T - 1) / T), 3, 1);
  k_cn_vel_f32<<<grd, T, 0, s>>>(f.u, f.ru, f.v, f.rv, f.w, f.rw, cell, face, g.nyc, P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 grd2((unsigned)((P + T - 1) / T), 2, 1);
  k_cn_ion_mixed<<<grd2, T, 0, s>>>(f.cp, reinterpret_cast<float*>(f.rcp), sh.cp, f.cm, reinterpret_cast<float*>(f.rcm),
                                    sh.cm, ion, R.Rref_p + (size_t)l * g.nyc, R.Rref_m + (size_t)l * g.nyc, R, g.nyc, P);
  return cudaGetLastError();
}

cudaError_t launch_plane_means3(const double* a, const double* b, const double* c, int nplanes, size_t P,
                                double* oa, double* ob, double* oc, cudaStream_t s) {
  k_plane_means3<<<nplanes, 256, 0, s>>>(a, b, c, P, oa, ob, oc);
  return cudaGetLastError();
}

cudaError_t launch_make_shadows(const double* cp, const double* cm, const double* Phi, const double* Hcp,
                                const double* Hcm, const Shadows& sh, const MixedRefs& R, const double* Href_p,
                                const double* Href_m, size_t P, size_t n, cudaStream_t s) {
  const int T = 256;
  k_make_shadows<<<(unsigned)((n + T - 1) / T), T, 0, s>>>(cp, cm, Phi, Hcp, Hcm, sh, R, Href_p, Href_m, P, n);
  return cudaGetLastError();
}

cudaError_t launch_from_shadow(const float* sh, const double* ref, double* out, size_t P, size_t n, cudaStream_t s) {
  const int T = 256;
  k_from_shadow<<<(unsigned)((n + T - 1) / T), T, 0, s>>>(sh, ref, out, P, n);
  return cudaGetLastError();
}

}  // namespace pnp
