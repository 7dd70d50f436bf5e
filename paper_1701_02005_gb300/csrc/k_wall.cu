// Wall-model data kernels: restriction of a fine state onto a coarse grid,
// near-wall feature columns of a state, training labels from a fine state,
// and the wall conditions that couple a wall model into the coarse solver
// (slip velocities or stresses, wall-potential offsets, ion-flux transfers).  (The paper resolves the double layer; the learned wall model that
// replaces it on a coarse y-grid has no counterpart in the paper.)
//
// Coarse grid: Nx_c = Nx_f / rx, Nz_c = Nz_f / rz, and every ry-th fine
// y-face is a coarse y-face.  A coarse value is the volume-weighted mean of
// the fine values whose indices map onto it (i_f = rx i_c + a, k_f = rz k_c + b,
// fine cells ry j_c .. ry j_c + ry - 1, weighted by their heights).
//
// Wall frame: a feature row belongs to one wall column; the top wall is
// mapped onto the bottom one by the rotation (x, y) -> (-x, -y) combined with
// c+ <-> c-, Phi -> -Phi, under which the plane Couette problem is invariant,
// so that one network serves both walls.  Streamwise velocities are taken
// relative to the wall: u_rel = u + Uw (bottom), Uw - u (top).
#include "pnp_common.cuh"
#include "pnp_wall.cuh"

namespace pnp {

template <typename T>
__device__ __forceinline__ double D(const T* p, size_t i) { return (double)p[i]; }

// Restrict one cell-centred (or x/z-face) field: out[jc][kc][ic].
template <typename T>
__global__ void k_restrict(const T* __restrict__ f, const double* __restrict__ dyf, WallMap wm, double* __restrict__ out) {
  const size_t n = (size_t)wm.nyc_c * wm.nz_c * wm.nx_c;
  const size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const int ic = (int)(o % wm.nx_c);
  const int kc = (int)((o / wm.nx_c) % wm.nz_c);
  const int jc = (int)(o / ((size_t)wm.nx_c * wm.nz_c));
  double acc = 0.0, vol = 0.0;
  for (int b = 0; b < wm.ry; ++b) {
    const int jf = jc * wm.ry + b;
    const double w = dyf[jf];
    double s = 0.0;
    for (int kk = 0; kk < wm.rz; ++kk)
      for (int ii = 0; ii < wm.rx; ++ii)
        s += D(f, cidx(jf, kc * wm.rz + kk, ic * wm.rx + ii, wm.nz_f, wm.nx_f));
    acc += w * s;
    vol += w * (wm.rx * wm.rz);
  }
  out[o] = acc / vol;
}

// Restrict v (y-faces): coarse face jc is fine face ry*jc; average over x/z.
template <typename T>
__global__ void k_restrict_v(const T* __restrict__ f, WallMap wm, double* __restrict__ out) {
  const size_t n = (size_t)(wm.nyc_c + 1) * wm.nz_c * wm.nx_c;
  const size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const int ic = (int)(o % wm.nx_c);
  const int kc = (int)((o / wm.nx_c) % wm.nz_c);
  const int jc = (int)(o / ((size_t)wm.nx_c * wm.nz_c));
  const int jf = jc * wm.ry;
  double s = 0.0;
  for (int kk = 0; kk < wm.rz; ++kk)
    for (int ii = 0; ii < wm.rx; ++ii) s += D(f, cidx(jf, kc * wm.rz + kk, ic * wm.rx + ii, wm.nz_f, wm.nx_f));
  out[o] = s / (wm.rx * wm.rz);
}

// Feature rows: [wall][k][i] x [field][d], d = 0..ncells-1 cells away from the wall.
template <typename TV>
__global__ void k_wall_features(const TV* __restrict__ u, const TV* __restrict__ w, IonView ions,
                                const double* __restrict__ yc, Geo g, double V, double Uw, int ncells,
                                const double* __restrict__ lift, float* __restrict__ X) {
  const size_t P = (size_t)g.nz * g.nx;
  const size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= 2 * P) return;
  const int wall = (int)(r / P);
  const size_t col = r - (size_t)wall * P;
  float* row = X + r * (size_t)(5 * ncells);
  for (int d = 0; d < ncells; ++d) {
    const int j = wall == 0 ? d : g.nyc - 1 - d;
    const size_t o = (size_t)j * P + col;
    const double phi = ions.phv(j, o) - V * yc[j] - (lift ? lift[o] : 0.0);
    const double ur = wall == 0 ? (double)u[o] + Uw : Uw - (double)u[o];
    const double cpo = ions.cpv(j, o), cmo = ions.cmv(j, o);
    row[0 * ncells + d] = (float)ur;
    row[1 * ncells + d] = (float)(double)w[o];
    row[2 * ncells + d] = (float)(wall == 0 ? cpo : cmo);
    row[3 * ncells + d] = (float)(wall == 0 ? cmo : cpo);
    row[4 * ncells + d] = (float)(wall == 0 ? phi : -phi);
  }
}

// Labels of coarse wall column (wall, kc, ic) from the fine state:
//  0: filtered wall shear rate d(u_rel)/dy of the fine state (wall frame),
//  1: the same for w,
//  2: potential perturbation phi = Phi - V y of the first coarse cell (wall frame),
//  3, 4: total y-flux of the counter- and co-ion through the first interior coarse
//        face (wall frame: positive away from the wall).
template <typename TV>
__global__ void k_wall_labels(const TV* __restrict__ u, const TV* __restrict__ v, const TV* __restrict__ w,
                              IonView ions, const double* __restrict__ ycf,
                              const double* __restrict__ dyf, const double* __restrict__ hf, WallMap wm, double h0c,
                              double V, double Uw, double D_ion, float* __restrict__ T) {
  const size_t Pc = (size_t)wm.nz_c * wm.nx_c;
  const size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= 2 * Pc) return;
  const int wall = (int)(r / Pc);
  const int ic = (int)(r % wm.nx_c);
  const int kc = (int)((r / wm.nx_c) % wm.nz_c);
  const int nycf = wm.nyc_f;
  const size_t Pf = (size_t)wm.nz_f * wm.nx_f;
  // restricted first coarse cell values (fine cells 0..ry-1 from the wall), wall frame
  double ua = 0.0, wa = 0.0, pa = 0.0, vol = 0.0;
  double gu = 0.0, gw = 0.0;   // fine wall gradients, averaged
  double fpl = 0.0, fmi = 0.0; // fine total ion fluxes through the coarse face, averaged
  const int jface = wall == 0 ? wm.ry : nycf - wm.ry;   // fine index of coarse face 1 (or nyc_c - 1)
  const double ihf = 1.0 / hf[jface];
  for (int kk = 0; kk < wm.rz; ++kk) {
    for (int ii = 0; ii < wm.rx; ++ii) {
      const int kf = kc * wm.rz + kk, i_f = ic * wm.rx + ii;
      const size_t col = (size_t)kf * wm.nx_f + i_f;
      for (int b = 0; b < wm.ry; ++b) {
        const int jf = wall == 0 ? b : nycf - 1 - b;
        const size_t o = (size_t)jf * Pf + col;
        const double wt = dyf[jf];
        ua += wt * (wall == 0 ? (double)u[o] + Uw : Uw - (double)u[o]);
        wa += wt * (double)w[o];
        const double phi = ions.phv(jf, o) - V * ycf[jf];
        pa += wt * (wall == 0 ? phi : -phi);
        vol += wt;
      }
      const int j0 = wall == 0 ? 0 : nycf - 1;
      const size_t o0 = (size_t)j0 * Pf + col;
      const double u0 = wall == 0 ? (double)u[o0] + Uw : Uw - (double)u[o0];
      gu += u0 / hf[wall == 0 ? 0 : nycf];
      gw += (double)w[o0] / hf[wall == 0 ? 0 : nycf];
      // total flux F = v c_f - D (dc/dy + s c_f dPhi/dy) on fine face jface (lab frame, +y)
      const size_t oa = (size_t)(jface - 1) * Pf + col, ob = (size_t)jface * Pf + col;
      const double vf = (double)v[(size_t)jface * Pf + col];
      const double cpa = ions.cpv(jface - 1, oa), cpb = ions.cpv(jface, ob);
      const double cma = ions.cmv(jface - 1, oa), cmb = ions.cmv(jface, ob);
      const double dP = (ions.phv(jface, ob) - ions.phv(jface - 1, oa)) * ihf;
      const double cpf = 0.5 * (cpa + cpb), cmf = 0.5 * (cma + cmb);
      const double Fp = vf * cpf - D_ion * ((cpb - cpa) * ihf + cpf * dP);
      const double Fm = vf * cmf - D_ion * ((cmb - cma) * ihf - cmf * dP);
      // wall frame: away from the wall is +y at the bottom, -y at the top; top swaps the ions
      if (wall == 0) { fpl += Fp; fmi += Fm; }
      else { fpl += -Fm; fmi += -Fp; }
    }
  }
  const double nrm = 1.0 / (wm.rx * wm.rz);
  ua /= vol;
  wa /= vol;
  pa /= vol;
  gu *= nrm;
  gw *= nrm;
  float* t = T + r * 5;
  t[0] = (float)gu;
  t[1] = (float)gw;
  (void)ua;
  (void)wa;
  (void)h0c;
  t[2] = (float)pa;
  t[3] = (float)(fpl * nrm);
  t[4] = (float)(fmi * nrm);
}

// Wall velocities (lab frame) from model outputs Y[wall][k][i][5] (wall-frame
// slips).  A slip that is not finite or exceeds ten wall speeds in magnitude
// falls back to the no-slip wall of the resolved method.
__device__ __forceinline__ double guard_slip(float s, double lim) {
  return (isfinite(s) && fabs((double)s) <= lim) ? (double)s : 0.0;
}

// The model predicts the wall shear rates g_u, g_w of a column; the wall slip
// that makes the coarse wall shear equal to them is s = q_0 - h_0 g, with q_0
// the coarse first-cell value (feature column 0 for u_rel, ncells for w) and
// h_0 the wall-to-centre distance.
template <typename TV>
__global__ void k_set_slip(const float* __restrict__ X, int ncells, const float* __restrict__ Y, size_t P, double Uw,
                           double h0b, double h0t, TV* __restrict__ wall_u, TV* __restrict__ wall_w) {
  const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P) return;
  const size_t fs = (size_t)5 * ncells;
  const float* xb = X + c * fs;
  const float* xt = X + (P + c) * fs;
  const float* yb = Y + c * 5;
  const float* yt = Y + (P + c) * 5;
  const double lim = 10.0 * (fabs(Uw) > 0.0 ? fabs(Uw) : 1.0);
  const float sub = (float)((double)xb[0] - h0b * (double)yb[0]);
  const float sut = (float)((double)xt[0] - h0t * (double)yt[0]);
  const float swb = (float)((double)xb[ncells] - h0b * (double)yb[1]);
  const float swt = (float)((double)xt[ncells] - h0t * (double)yt[1]);
  wall_u[c] = (TV)(guard_slip(sub, lim) - Uw);       // bottom: u = u_rel - Uw
  wall_u[P + c] = (TV)(Uw - guard_slip(sut, lim));   // top: u = Uw - u_rel
  wall_w[c] = (TV)guard_slip(swb, lim);
  wall_w[P + c] = (TV)guard_slip(swt, lim);
}

// Under-relaxed wall-shear rates: prev += w (Y - prev) for the two rate
// columns of every row, and Y takes the relaxed value.
__global__ void k_relax_rates(float* __restrict__ Y, float* __restrict__ prev, int rows, float w) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const size_t o = (size_t)r * 5 + q;
    const float v = prev[o] + w * (Y[o] - prev[o]);
    prev[o] = v;
    Y[o] = v;
  }
}

// Plane means of the two wall-shear-rate columns of each wall's rows (rows
// [0, P) bottom, [P, 2P) top) over the rows with finite predictions, written
// back to every row of that wall.
__global__ void k_mean_rates(float* __restrict__ Y, int P) {
  __shared__ float sh[3][256];
  const int wall = blockIdx.x;
  float a = 0.f, b = 0.f, n = 0.f;
  for (int r = threadIdx.x; r < P; r += blockDim.x) {
    const float ya = Y[(size_t)(wall * P + r) * 5 + 0], yb = Y[(size_t)(wall * P + r) * 5 + 1];
    if (isfinite(ya) && isfinite(yb)) {   // a non-finite prediction does not enter the mean
      a += ya;
      b += yb;
      n += 1.f;
    }
  }
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  sh[2][threadIdx.x] = n;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + st];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + st];
      sh[2][threadIdx.x] += sh[2][threadIdx.x + st];
    }
    __syncthreads();
  }
  // no finite row: NaN, which the wall-value kernel turns into the no-slip wall
  const float cnt = sh[2][0];
  const float ma = cnt > 0.f ? sh[0][0] / cnt : __int_as_float(0x7fc00000);
  const float mb = cnt > 0.f ? sh[1][0] / cnt : __int_as_float(0x7fc00000);
  for (int r = threadIdx.x; r < P; r += blockDim.x) {
    Y[(size_t)(wall * P + r) * 5 + 0] = ma;
    Y[(size_t)(wall * P + r) * 5 + 1] = mb;
  }
}

cudaError_t launch_mean_rates(float* Y, int P, cudaStream_t s) {
  k_mean_rates<<<2, 256, 0, s>>>(Y, P);
  return cudaGetLastError();
}

cudaError_t launch_relax_rates(float* Y, float* prev, int rows, float w, cudaStream_t s) {
  k_relax_rates<<<(rows + 255) / 256, 256, 0, s>>>(Y, prev, rows, w);
  return cudaGetLastError();
}

// Potential coupling: the wall-potential offsets (lab frame, relative to the
// uniform walls -V, +V) move by gain (phi_pred - phi_1) per call, phi_pred the
// network's first-cell potential (column 2, wall frame: the top wall's sign is
// flipped back) and phi_1 the first cell's present potential perturbation: the
// feature row's value, which leaves out the charge-free lift of the offsets, plus
// that lift (lift: its first and last cell planes, or null when there is none).
// Offsets stay within +-lim; a non-finite prediction leaves the offset alone.
__global__ void k_edl_offsets(const float* __restrict__ X, int ncells, const float* __restrict__ Y, size_t P,
                              double gain, double lim, const double* __restrict__ lift, int nyc,
                              double* __restrict__ B, double* __restrict__ T) {
  const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P) return;
  const size_t fs = (size_t)5 * ncells;
  const double lb = lift ? lift[c] : 0.0, lt = lift ? -lift[(size_t)(nyc - 1) * P + c] : 0.0;   // wall frame
  const double db = gain * ((double)Y[c * 5 + 2] - ((double)X[c * fs + 4 * ncells] + lb));
  const double dt = gain * ((double)Y[(P + c) * 5 + 2] - ((double)X[(P + c) * fs + 4 * ncells] + lt));
  if (isfinite(db)) B[c] = fmin(fmax(B[c] + db, -lim), lim);
  if (isfinite(dt)) T[c] = fmin(fmax(T[c] - dt, -lim), lim);
}

// Ion-flux coupling: the total ion fluxes through the first interior face of
// each wall column (face 1 at the bottom, face Nyc-1 at the top) are moved a
// fraction gain of the way to the predicted ones (columns 3, 4, wall frame) by
// transferring ions between the two cells that share the face, over dt:
// conservative per column.  The transfer out of a cell is limited to half its
// content; the flux of the state is the discrete one of the labels,
// F = v c_f - D (dc/dy + s c_f dPhi/dy), c_f the face mean.  With the df
// shadows of a mixed-precision context (S != null) the corrected cells'
// shadows are rewritten from the FP64 values.
template <typename TV>
__global__ void k_wall_flux_fix(IonView ions, const TV* __restrict__ v, const double* __restrict__ idy,
                                const double* __restrict__ ih, Geo g, double Dion, const float* __restrict__ Y,
                                double gain, double dt) {
  const size_t P = (size_t)g.nz * g.nx;
  const size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= 2 * P) return;
  const int wall = (int)(r / P);
  const size_t col = r - (size_t)wall * P;
  const int jl = wall == 0 ? 0 : g.nyc - 2, ju = jl + 1, jf = jl + 1;   // cells below / above face jf
  const size_t ol = (size_t)jl * P + col, ou = (size_t)ju * P + col;
  const double ihf = ih[jf];
  const double vf = (double)v[(size_t)jf * P + col];
  const double dP = (ions.phv(ju, ou) - ions.phv(jl, ol)) * ihf;
  double cp[2] = {ions.cpv(jl, ol), ions.cpv(ju, ou)}, cm[2] = {ions.cmv(jl, ol), ions.cmv(ju, ou)};
  const double cpf = 0.5 * (cp[0] + cp[1]), cmf = 0.5 * (cm[0] + cm[1]);
  const double Fp = vf * cpf - Dion * ((cp[1] - cp[0]) * ihf + cpf * dP);
  const double Fm = vf * cmf - Dion * ((cm[1] - cm[0]) * ihf - cmf * dP);
  const float* y = Y + r * 5;
  // wall frame -> lab frame (+y): the top wall's counter-ion column is c-, fluxes flip sign
  double dFp, dFm;
  if (wall == 0) {
    dFp = gain * ((double)y[3] - Fp);
    dFm = gain * ((double)y[4] - Fm);
  } else {
    dFm = -gain * ((double)y[3] + Fm);
    dFp = -gain * ((double)y[4] + Fp);
  }
  auto apply = [&](double (&c)[2], double dF, double* c64, float* S, float* L, const double* cref) {
    if (!isfinite(dF)) return;
    // the cell that loses ions gives at most half of them
    const double cap = dF > 0.0 ? 0.5 * fmax(c[0], 0.0) / (idy[jl] * dt) : 0.5 * fmax(c[1], 0.0) / (idy[ju] * dt);
    dF = fmin(fmax(dF, -cap), cap);
    c[0] -= dF * dt * idy[jl];
    c[1] += dF * dt * idy[ju];
    if (c64) {
      c64[ol] = c[0];
      c64[ou] = c[1];
    } else {
      const double a = c[0] - cref[jl], b = c[1] - cref[ju];
      S[ol] = (float)a;
      L[ol] = (float)(a - (double)S[ol]);
      S[ou] = (float)b;
      L[ou] = (float)(b - (double)S[ou]);
    }
  };
  apply(cp, dFp, const_cast<double*>(ions.cp), const_cast<float*>(ions.cpS), const_cast<float*>(ions.cpL),
        ions.crefp);
  apply(cm, dFm, const_cast<double*>(ions.cm), const_cast<float*>(ions.cmS), const_cast<float*>(ions.cmL),
        ions.crefm);
}

cudaError_t launch_edl_offsets(const float* X, int ncells, const float* Y, size_t P, double gain, double lim,
                               const double* lift, int nyc, double* B, double* T, cudaStream_t s) {
  k_edl_offsets<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(X, ncells, Y, P, gain, lim, lift, nyc, B, T);
  return cudaGetLastError();
}

template <typename TV>
cudaError_t launch_wall_flux_fix(const IonView& ions, const TV* v, const double* idy, const double* ih, const Geo& g,
                                 double Dion, const float* Y, double gain, double dt, cudaStream_t s) {
  const size_t n = 2 * (size_t)g.nz * g.nx;
  k_wall_flux_fix<TV><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(ions, v, idy, ih, g, Dion, Y, gain, dt);
  return cudaGetLastError();
}

// ---- launchers ----
template <typename T>
cudaError_t launch_restrict(const T* f, const double* dyf, const WallMap& wm, double* out, bool vfield, cudaStream_t s) {
  const int B = 256;
  if (vfield) {
    const size_t n = (size_t)(wm.nyc_c + 1) * wm.nz_c * wm.nx_c;
    k_restrict_v<T><<<(unsigned)((n + B - 1) / B), B, 0, s>>>(f, wm, out);
  } else {
    const size_t n = (size_t)wm.nyc_c * wm.nz_c * wm.nx_c;
    k_restrict<T><<<(unsigned)((n + B - 1) / B), B, 0, s>>>(f, dyf, wm, out);
  }
  return cudaGetLastError();
}

template <typename TV>
cudaError_t launch_wall_features(const TV* u, const TV* w, const IonView& ions, const double* yc, const Geo& g,
                                 double V, double Uw, int ncells, const double* lift, float* X, cudaStream_t s) {
  const size_t n = 2 * (size_t)g.nz * g.nx;
  k_wall_features<TV><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(u, w, ions, yc, g, V, Uw, ncells, lift, X);
  return cudaGetLastError();
}

template <typename TV>
cudaError_t launch_wall_labels(const TV* u, const TV* v, const TV* w, const IonView& ions, const double* ycf,
                               const double* dyf, const double* hf, const WallMap& wm, double h0c, double V,
                               double Uw, double D_ion, float* T, cudaStream_t s) {
  const size_t n = 2 * (size_t)wm.nz_c * wm.nx_c;
  k_wall_labels<TV><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(u, v, w, ions, ycf, dyf, hf, wm, h0c, V, Uw, D_ion,
                                                               T);
  return cudaGetLastError();
}

template <typename TV>
cudaError_t launch_set_slip(const float* X, int ncells, const float* Y, size_t P, double Uw, double h0b, double h0t,
                            TV* wall_u, TV* wall_w, cudaStream_t s) {
  k_set_slip<TV><<<(unsigned)((P + 255) / 256), 256, 0, s>>>(X, ncells, Y, P, Uw, h0b, h0t, wall_u, wall_w);
  return cudaGetLastError();
}

template cudaError_t launch_restrict<double>(const double*, const double*, const WallMap&, double*, bool, cudaStream_t);
template cudaError_t launch_restrict<float>(const float*, const double*, const WallMap&, double*, bool, cudaStream_t);
template cudaError_t launch_wall_features<double>(const double*, const double*, const IonView&, const double*,
                                                  const Geo&, double, double, int, const double*, float*,
                                                  cudaStream_t);
template cudaError_t launch_wall_features<float>(const float*, const float*, const IonView&, const double*,
                                                 const Geo&, double, double, int, const double*, float*,
                                                 cudaStream_t);
template cudaError_t launch_wall_labels<double>(const double*, const double*, const double*, const IonView&,
                                                const double*, const double*, const double*, const WallMap&, double,
                                                double, double, double, float*, cudaStream_t);
template cudaError_t launch_wall_labels<float>(const float*, const float*, const float*, const IonView&, const double*,
                                               const double*, const double*, const WallMap&, double, double, double,
                                               double, float*, cudaStream_t);
template cudaError_t launch_wall_flux_fix<double>(const IonView&, const double*, const double*, const double*,
                                                  const Geo&, double, const float*, double, double, cudaStream_t);
template cudaError_t launch_wall_flux_fix<float>(const IonView&, const float*, const double*, const double*,
                                                 const Geo&, double, const float*, double, double, cudaStream_t);
template cudaError_t launch_set_slip<double>(const float*, int, const float*, size_t, double, double, double, double*,
                                             double*, cudaStream_t);
template cudaError_t launch_set_slip<float>(const float*, int, const float*, size_t, double, double, double, float*,
                                            float*, cudaStream_t);

}  // namespace pnp
