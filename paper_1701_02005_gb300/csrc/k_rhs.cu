// Explicit right-hand sides of one RK3 substage (arXiv:1701.02005, Eq. (1)
// momentum with the Coulomb force, Eq. (3) Nernst-Planck for c+ and c-,
// staggered as in Fig. 1; Numerical methods for the time integration).
//
// One thread owns one cell (i, j, k) and produces, for the u point on its
// x-face i, the w point on its z-face k, the v point on its bottom y-face j
// (j >= 1) and the two ion concentrations at its centre:
//   H  = -div(flux) + x/z diffusion + body force        (explicit terms)
//   r  = dt [gam H + zet H_old - alp G p + alp nu L_y q] (Crank-Nicolson RHS)
// H overwrites H_old in place (each thread touches only its own entries).
#include "pnp_common.cuh"

namespace pnp {

template <typename T>
__device__ __forceinline__ double L(const T* p, size_t i) {
  return (double)__ldg(p + i);
}

template <typename TV>
__global__ void __launch_bounds__(128) k_rhs(Fields<TV> f, Geo g, Metrics mt, Phys ph, Stage st) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.z;
  if (i >= g.nx || k >= g.nz) return;
  const int nx = g.nx, nz = g.nz, nyc = g.nyc;
  const int im = i ? i - 1 : nx - 1, ip = (i + 1 == nx) ? 0 : i + 1;
  const int km = k ? k - 1 : nz - 1, kp = (k + 1 == nz) ? 0 : k + 1;
  const bool has_dn = j > 0, has_up = j < nyc - 1;
  const double idx = g.idx, idz = g.idz;
  const double idx2 = idx * idx, idz2 = idz * idz;
  const size_t c0 = cidx(j, k, i, nz, nx);
  const size_t cxm = cidx(j, k, im, nz, nx), cxp = cidx(j, k, ip, nz, nx);
  const size_t czm = cidx(j, km, i, nz, nx), czp = cidx(j, kp, i, nz, nx);
  const size_t P = (size_t)nz * nx;
  const double idyj = mt.idy[j];

  // ---------------- shared loads ----------------
  const double u0 = L(f.u, c0), uxm = L(f.u, cxm), uxp = L(f.u, cxp), uzm = L(f.u, czm), uzp = L(f.u, czp);
  const double uym = has_dn ? L(f.u, c0 - P) : 0.0, uyp = has_up ? L(f.u, c0 + P) : 0.0;
  const double w0 = L(f.w, c0), wxm = L(f.w, cxm), wxp = L(f.w, cxp), wzm = L(f.w, czm), wzp = L(f.w, czp);
  const double wym = has_dn ? L(f.w, c0 - P) : 0.0, wyp = has_up ? L(f.w, c0 + P) : 0.0;
  // v on the bottom face j and top face j+1 of this cell (wall faces hold zeros)
  const double vb = L(f.v, c0), vt = L(f.v, c0 + P);
  const double Ph0 = L(f.Phi, c0), Phxm = L(f.Phi, cxm), Phxp = L(f.Phi, cxp);
  const double Phzm = L(f.Phi, czm), Phzp = L(f.Phi, czp);
  const double Phym = has_dn ? L(f.Phi, c0 - P) : 0.0, Phyp = has_up ? L(f.Phi, c0 + P) : 0.0;
  const double cp0 = L(f.cp, c0), cm0 = L(f.cm, c0);
  const double rho0 = cp0 - cm0;
  const double p0 = L(f.p, c0);

  // ---------------- u at (x-face i, y-centre j, z-centre k) ----------------
  {
    const double ubp = 0.5 * (u0 + uxp), ubm = 0.5 * (uxm + u0);
    const double ax = (ubp * ubp - ubm * ubm) * idx;
    const double vft = 0.5 * (L(f.v, cidx(j + 1, k, im, nz, nx)) + vt);   // v at (x-face i, y-face j+1)
    const double vfb = 0.5 * (L(f.v, cxm) + vb);                 // v at (x-face i, y-face j)
    const double uft = has_up ? 0.5 * (u0 + uyp) : 0.0;
    const double ufb = has_dn ? 0.5 * (uym + u0) : 0.0;
    const double ay = (vft * uft - vfb * ufb) * idyj;
    const double wfk = 0.5 * (wxm + w0);                        // w at (x-face i, z-face k)
    const double wfkp = 0.5 * (L(f.w, cidx(j, kp, im, nz, nx)) + wzp);   // w at (x-face i, z-face k+1)
    const double az = (wfkp * 0.5 * (u0 + uzp) - wfk * 0.5 * (uzm + u0)) * idz;
    const double lap = (uxp - 2.0 * u0 + uxm) * idx2 + (uzp - 2.0 * u0 + uzm) * idz2;
    const double rhom = L(f.cp, cxm) - L(f.cm, cxm);
    const double fu = -ph.K * 0.5 * (rhom + rho0) * (Ph0 - Phxm) * idx;
    const double H = -(ax + ay + az) + (st.af ? 0.0 : ph.nu * lap) + fu;
    const double ub = f.wall_u ? (double)f.wall_u[(size_t)k * nx + i] : -ph.Uw;
    const double ut = f.wall_u ? (double)f.wall_u[P + (size_t)k * nx + i] : ph.Uw;
    const double Ly = mt.lo_c[j] * ((has_dn ? uym : ub) - u0) + mt.hi_c[j] * ((has_up ? uyp : ut) - u0);
    const double gp = (p0 - L(f.p, cxm)) * idx;
    const double Ho = (double)f.Hu[c0];
    f.ru[c0] = (TV)(st.dt * (st.gam * H + st.zet * Ho - st.alp * gp + st.alp * ph.nu * (st.af ? Ly + lap : Ly)));
    f.Hu[c0] = (TV)H;
  }

  // ---------------- w at (x-centre i, y-centre j, z-face k) ----------------
  {
    const double wbp = 0.5 * (w0 + wzp), wbm = 0.5 * (wzm + w0);
    const double az = (wbp * wbp - wbm * wbm) * idz;
    const double vft = 0.5 * (L(f.v, cidx(j + 1, km, i, nz, nx)) + vt);
    const double vfb = 0.5 * (L(f.v, czm) + vb);
    const double wft = has_up ? 0.5 * (w0 + wyp) : 0.0;
    const double wfb = has_dn ? 0.5 * (wym + w0) : 0.0;
    const double ay = (vft * wft - vfb * wfb) * idyj;
    const double ufi = 0.5 * (uzm + u0);                        // u at (x-face i, z-face k)
    const double ufip = 0.5 * (L(f.u, cidx(j, km, ip, nz, nx)) + uxp);   // u at (x-face i+1, z-face k)
    const double ax = (ufip * 0.5 * (w0 + wxp) - ufi * 0.5 * (wxm + w0)) * idx;
    const double lap = (wxp - 2.0 * w0 + wxm) * idx2 + (wzp - 2.0 * w0 + wzm) * idz2;
    const double rhom = L(f.cp, czm) - L(f.cm, czm);
    const double fw = -ph.K * 0.5 * (rhom + rho0) * (Ph0 - Phzm) * idz;
    const double H = -(ax + ay + az) + (st.af ? 0.0 : ph.nu * lap) + fw;
    const double wb = f.wall_w ? (double)f.wall_w[(size_t)k * nx + i] : 0.0;
    const double wt = f.wall_w ? (double)f.wall_w[P + (size_t)k * nx + i] : 0.0;
    const double Ly = mt.lo_c[j] * ((has_dn ? wym : wb) - w0) + mt.hi_c[j] * ((has_up ? wyp : wt) - w0);
    const double gp = (p0 - L(f.p, czm)) * idz;
    const double Ho = (double)f.Hw[c0];
    f.rw[c0] = (TV)(st.dt * (st.gam * H + st.zet * Ho - st.alp * gp + st.alp * ph.nu * (st.af ? Ly + lap : Ly)));
    f.Hw[c0] = (TV)H;
  }

  // ---------------- v at (x-centre i, y-face j, z-centre k), 1 <= j <= nyc-1 ----------------
  if (has_dn) {
    const double wl = mt.wl[j], wu = mt.wu[j], ihj = mt.ih[j];
    const size_t d0 = c0 - P;   // cell j-1
    const double v0 = vb;
    const double vxm = L(f.v, cxm), vxp = L(f.v, cxp), vzm = L(f.v, czm), vzp = L(f.v, czp);
    const double vym = L(f.v, c0 - P), vyp = vt;
    const double Ui = wl * L(f.u, d0) + wu * u0;                               // u at (x-face i, y-face j)
    const double Uip = wl * L(f.u, cidx(j - 1, k, ip, nz, nx)) + wu * uxp;     // u at (x-face i+1, y-face j)
    const double ax = (Uip * 0.5 * (v0 + vxp) - Ui * 0.5 * (vxm + v0)) * idx;
    const double vbu = 0.5 * (v0 + vyp), vbd = 0.5 * (vym + v0);
    const double ay = (vbu * vbu - vbd * vbd) * ihj;
    const double Wk = wl * L(f.w, d0) + wu * w0;                               // w at (y-face j, z-face k)
    const double Wkp = wl * L(f.w, cidx(j - 1, kp, i, nz, nx)) + wu * wzp;   // w at (y-face j, z-face k+1)
    const double az = (Wkp * 0.5 * (v0 + vzp) - Wk * 0.5 * (vzm + v0)) * idz;
    const double lap = (vxp - 2.0 * v0 + vxm) * idx2 + (vzp - 2.0 * v0 + vzm) * idz2;
    const double rhod = L(f.cp, d0) - L(f.cm, d0);
    const double fv = -ph.K * 0.5 * (rhod + rho0) * (Ph0 - Phym) * ihj;
    const double H = -(ax + ay + az) + (st.af ? 0.0 : ph.nu * lap) + fv;
    const double Ly = mt.lo_f[j] * (vym - v0) + mt.hi_f[j] * (vyp - v0);
    const double gp = (p0 - L(f.p, d0)) * ihj;
    const double Ho = (double)f.Hv[c0];
    f.rv[c0] = (TV)(st.dt * (st.gam * H + st.zet * Ho - st.alp * gp + st.alp * ph.nu * (st.af ? Ly + lap : Ly)));
    f.Hv[c0] = (TV)H;
  }

  // ---------------- c+ and c- at the cell centre (Eq. (3)) ----------------
  {
    const double D = ph.D;
    const double ux_i = u0, ux_ip = uxp;       // u on x-faces i and i+1
    const double wz_k = w0, wz_kp = wzp;       // w on z-faces k and k+1
    const double ihj = mt.ih[j], ihjp = mt.ih[j + 1];
#pragma unroll
    for (int ion = 0; ion < 2; ++ion) {
      const double* c = ion == 0 ? f.cp : f.cm;
      const double s = ion == 0 ? 1.0 : -1.0;
      const double cc = ion == 0 ? cp0 : cm0;
      const double cxm_ = L(c, cxm), cxp_ = L(c, cxp), czm_ = L(c, czm), czp_ = L(c, czp);
      const double cym_ = has_dn ? L(c, c0 - P) : 0.0, cyp_ = has_up ? L(c, c0 + P) : 0.0;
      // face fluxes F = u c_face - D grad c - s D c_face grad Phi
      double ca = 0.5 * (cxm_ + cc), cb = 0.5 * (cc + cxp_);
      const double Fx_i = ux_i * ca - D * (cc - cxm_) * idx - s * D * ca * (Ph0 - Phxm) * idx;
      const double Fx_ip = ux_ip * cb - D * (cxp_ - cc) * idx - s * D * cb * (Phxp - Ph0) * idx;
      ca = 0.5 * (czm_ + cc);
      cb = 0.5 * (cc + czp_);
      const double Fz_k = wz_k * ca - D * (cc - czm_) * idz - s * D * ca * (Ph0 - Phzm) * idz;
      const double Fz_kp = wz_kp * cb - D * (czp_ - cc) * idz - s * D * cb * (Phzp - Ph0) * idz;
      // y faces: advection + migration only (y diffusion is implicit); walls carry no flux
      double Fy_j = 0.0, Fy_jp = 0.0;
      if (has_dn) {
        const double cf = 0.5 * (cym_ + cc);
        Fy_j = vb * cf - s * D * cf * (Ph0 - Phym) * ihj;
      }
      if (has_up) {
        const double cf = 0.5 * (cc + cyp_);
        Fy_jp = vt * cf - s * D * cf * (Phyp - Ph0) * ihjp;
      }
      double H = -((Fx_ip - Fx_i) * idx + (Fy_jp - Fy_j) * idyj + (Fz_kp - Fz_k) * idz);
      double Ly = (has_dn ? mt.lo_c[j] * (cym_ - cc) : 0.0) + (has_up ? mt.hi_c[j] * (cyp_ - cc) : 0.0);
      if (st.af) {   // the x/z diffusion leaves H and joins the implicit operator
        const double lapc = (cxp_ - 2.0 * cc + cxm_) * idx2 + (czp_ - 2.0 * cc + czm_) * idz2;
        H -= D * lapc;
        Ly += lapc;
      }
      double* Hc = ion == 0 ? f.Hcp : f.Hcm;
      double* rc = ion == 0 ? f.rcp : f.rcm;
      const double Ho = Hc[c0];
      rc[c0] = st.dt * (st.gam * H + st.zet * Ho + st.alp * D * Ly);
      Hc[c0] = H;
    }
  }
}

template <typename TV>
cudaError_t launch_rhs(const Fields<TV>& f, const Geo& g, const Metrics& m, const Phys& ph,
                       const Stage& st, cudaStream_t s) {
  const int bx = g.lc_rhs_bx ? g.lc_rhs_bx : 32, by = 128 / bx;
  dim3 blk(bx, by, 1);
  dim3 grd((g.nx + bx - 1) / bx, (g.nz + by - 1) / by, g.nyc);
  k_rhs<TV><<<grd, blk, 0, s>>>(f, g, m, ph, st);
  return cudaGetLastError();
}

template cudaError_t launch_rhs<double>(const Fields<double>&, const Geo&, const Metrics&, const Phys&,
                                        const Stage&, cudaStream_t);
template cudaError_t launch_rhs<float>(const Fields<float>&, const Geo&, const Metrics&, const Phys&,
                                       const Stage&, cudaStream_t);

}  // namespace pnp
