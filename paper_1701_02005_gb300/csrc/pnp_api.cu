// C ABI of libpnp (declared in include/pnp.h): context set-up, workspace
// carving, host-side precomputation of grid metrics / elimination factors /
// FFT tables, and the orchestration of one fractional step
// (arXiv:1701.02005, Numerical methods):
//   per RK3 substage l:  explicit terms -> y-implicit CN solves ->
//   pressure Poisson (Neumann) + projection -> potential Poisson (Dirichlet).
// A step is captured once per dt into a CUDA graph on non-default streams.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "pnp_common.cuh"
#include "pnp_mixed.cuh"
#include "pnp_df.cuh"
#include "pnp_wall.cuh"

using namespace pnp;

namespace {

// Low-storage RK3 coefficients (Rai & Moin 1991); alpha = gamma + zeta.
const double kGam[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
const double kZet[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};

constexpr size_t kAlign = 256;
// CN factor-row families: 0 u, w (Dirichlet wall values); 1 v (interior faces);
// 2 ions (zero wall flux, D); 3 u, w with a prescribed wall stress (zero wall
// coupling in the implicit operator, nu) for the wall model's stress coupling
constexpr int kCnKinds = 4;
constexpr int kDiagBlocks = 760;   // 5 x 152 SMs of 256-thread blocks: one resident wave
constexpr int kProbeBlocks = 152 * 8;

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

struct Bump {
  char* base;
  size_t off = 0;
  template <typename T> T* take(size_t count) {
    off = (off + kAlign - 1) / kAlign * kAlign;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

}  // namespace

// Optional per-launch-site event timing (pnp_profile).
struct Prof {
  static constexpr int kMax = 64;
  cudaEvent_t ev[kMax];
  int site[kMax], on_aux[kMax];
  int n = 0;
  bool timeline = false;   // record on each site's own stream, keep the concurrent schedule
  bool external = false;   // during a stream capture: record as event nodes of the graph
};

struct pnp_ctx {
  Prof* prof = nullptr;
  Geo g{};
  int precision = PNP_FP64;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  size_t nc = 0, nv = 0;
  // prognostic + work fields; velocity-type arrays are double (FP64) or float (MIXED)
  void *u, *v, *w, *p, *Hu, *Hv, *Hw, *ru, *rv, *rw;
  double *cp, *cm, *Phi, *Hcp, *Hcm, *rcp, *rcm;
  double* sreal;   // real scratch: Phi_p, spectral elimination multipliers
  void* spec;      // spectral buffer, (nyc, nz, mp) complex (FP64-sized)
  double* stage;   // conversion staging, nv values
  // per-y metrics (device) and their host copies
  double *yf_d, *yc_d, *idy_d, *ih_d, *lo_c_d, *hi_c_d, *lo_f_d, *hi_f_d, *wl_d, *wu_d;
  double *kx2_d, *kz2_d;
  double *rowsN_d, *rowsD_d;   // a, b, c of the Neumann / Dirichlet y-operator (3 * nyc)
  double* cn_d;                // [3 substages][3 kinds][a, c, m][ny]
  void *twx_d, *twp_d, *twz_d;      // complex<double> tables
  void *twx_f, *twp_f, *twz_f;      // complex<float> tables
  double* diag_partial;
  double* diag_out;
  int* status_d;
  double* probe_d;
  // mixed-precision path: FP32 shadows, FP32 metrics / velocity CN rows, reference profiles
  float *cpS, *cmS, *phiS, *HcpS, *HcmS;
  float* mf[8];      // idy, ih, lo_c, hi_c, lo_f, hi_f, wl, wu
  float2* diag_w = nullptr;            // dy_j, h_j, 1/dy_j ([ny] each) as df pairs (mixed diagnostics)
  double refN_p = 0.0, refN_m = 0.0;   // sum over cells of c_ref(j) dy_j (reference part of N+-)
  float* cnF_d;      // [3 substages][3 kinds][a, c, m][ny]
  float *crefp_f, *crefm_f, *crfp_f, *crfm_f, *rhoref_f, *rhorf_f, *dPref_f, *Fvref_f;
  double *Rrefp_d, *Rrefm_d, *cref64p_d, *cref64m_d, *Phiref64_d, *meanrhs_d, *meanshift_d, *delta_d;
  double *Hrefp_d, *Hrefm_d;
  // spectral elimination factors (grid-only): c'_j and 1/pivot_j per spectral point
  double *spc_cprN, *spc_invN, *spc_cprD, *spc_invD;
  // mixed path: their double-float copies and the y-operator sub-diagonals as df
  float2 *spf_cprN = nullptr, *spf_invN = nullptr, *spf_cprD = nullptr, *spf_invD = nullptr;
  float2 *spf_aN = nullptr, *spf_aD = nullptr;
  // mixed path: low parts of the ion fluctuations (c = c_ref + S + L, S the shadow)
  float *cpL = nullptr, *cmL = nullptr;
  float2 *dCp_f2 = nullptr, *dCm_f2 = nullptr;   // [3][ny] reference increments as df pairs
  // mixed path: TMA descriptors of the stencil inputs (built once the workspace is carved)
  RhsMaps rhs_maps{};
  bool rhs_maps_ok = false;
  cplx<double>* dscr;   // FP64 forward-sweep values of the spectral solves
  // the potential pipeline runs concurrently with the pressure pipeline on an
  // auxiliary stream, with its own spectral buffers
  void* spec2 = nullptr;
  cplx<double>* dscr2 = nullptr;
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // wall model: per-column wall velocities [2][P] (velocity precision), feature / output rows
  void *wall_u, *wall_w;
  float *featX, *featY;
  bool slip_on = false;
  // wall-model coupling: 0 slip (the slip velocity is a Dirichlet wall value of
  // the implicit solve), 1 stress (the wall flux it implies is imposed, the
  // implicit operator has no wall coupling); relaxation of the predicted rates
  bool wall_stress = false;
  int wm_mode = 0;
  float wm_relax = 1.f;
  bool wm_have_prev = false;
  float* featYprev = nullptr;
  // double-layer coupling: gains of the wall-potential offsets and of the ion-flux
  // transfers (0: off); edl_map: the wall-potential map holds the offsets
  double edl_phi_gain = 0.0, edl_flux_gain = 0.0;
  bool edl_map = false;
  std::vector<double> href_p, href_m, lyc_p, lyc_m;
  bool refs_valid = false;   // references and shadows match the FP64 fields
  bool fp64_fresh = true;    // FP64 c+-, Phi, Hc+- arrays are current (else the shadows are)
  double refs_dt = NAN;
  std::vector<double> yf, yc, dy, h, cn_h;
  Phys ph{};
  double Re = 0, lam = 0, Sc = 1, beta = 0.5;
  bool have_params = false, have_state = false;
  double time = 0.0;
  long long nstep = 0;
  double last_dt = 0.0;                         // size of the last step (0: none yet)
  int policy = PNP_POLICY_DEFAULT;              // mixed path: where the solves' FP64 accuracy comes from
  // wall potentials that vary along the walls: Phi = V y + wall_off + lift + phi
  bool wall_map = false;
  double wall_off = 0.0, V_set = 0.0;           // mean offset; the uniform V of pnp_set_params
  double *wallB_d = nullptr, *wallT_d = nullptr, *lift64 = nullptr;
  float* lift32 = nullptr;
  // approximate factorisation (x/z implicit): periodic-sweep factors
  // [3 substages][2 kinds: nu, D][2 dirs: x, z] x {c', m, q} and their scalars
  int scheme = PNP_SCHEME_CN;
  double *af_d = nullptr;
  float* af_f = nullptr;
  double af_sc[3][2][2][3] = {};
  // the sweeps as truncated circulant convolutions: taps g_0 .. g_kConvMaxK of
  // each inverse (substage, kind, direction) and the taps an FP32 / FP64 pass
  // needs (-1: more than kConvMaxK, the Thomas sweeps run instead)
  double af_g[3][2][2][kConvMaxK + 1] = {};
  int af_kf[3][2][2] = {}, af_kd[3][2][2] = {};
  double af_dt = NAN;
  // the CN forward elimination fused into the mixed stencil: chunk products G
  // [3 substages][3 kinds][ny] for the dt and chunk length they were made for
  bool fuse_cn = true;
  float* fuseG_d = nullptr;
  double fuse_dt = NAN;
  int fuse_jc = 0;
  // time statistics: plane means of q and q^2 summed over samples ([12][ny])
  double* stats_acc = nullptr;
  long long stats_n = 0;
  double cfl_max = 1.7320508075688772, dphi_max = 2.0;   // limits of the device checks
  double refH_p = 0.0, refH_m = 0.0;            // sum over cells of H_ref(j) dy_j (mixed)
  cudaGraphExec_t gexec = nullptr;
  double graph_dt = NAN;
  double cn_dt = NAN;
};

namespace {

size_t carve(pnp_ctx* c, char* base, int nx, int ny, int nz, int precision) {
  Bump b{base};
  const int nyc = ny - 1;
  const int mh = nx / 2 + 1;
  const int mp = (mh + 7) / 8 * 8;
  const size_t nc = (size_t)nyc * nz * nx, nv = (size_t)ny * nz * nx;
  const size_t tv = precision == PNP_FP64 ? sizeof(double) : sizeof(float);
  const size_t nspec = (size_t)nyc * nz * mp;
  auto vel = [&](size_t n) { return b.take<char>(n * tv); };
  void *u = vel(nc), *w = vel(nc), *p = vel(nc), *Hu = vel(nc), *Hw = vel(nc), *ru = vel(nc), *rw = vel(nc);
  void *v = vel(nv), *Hv = vel(nv), *rv = vel(nv);
  double *cp = b.take<double>(nc), *cm = b.take<double>(nc), *Phi = b.take<double>(nc);
  double *Hcp = b.take<double>(nc), *Hcm = b.take<double>(nc), *rcp = b.take<double>(nc), *rcm = b.take<double>(nc);
  double* sreal = b.take<double>(nspec > nc ? nspec : nc);
  void* spec = b.take<cplx<double>>(nspec);
  double* stage = b.take<double>(nv);
  double *yf = b.take<double>(ny), *yc = b.take<double>(ny), *idy = b.take<double>(ny), *ih = b.take<double>(ny);
  double *lo_c = b.take<double>(ny), *hi_c = b.take<double>(ny), *lo_f = b.take<double>(ny), *hi_f = b.take<double>(ny);
  double *wl = b.take<double>(ny), *wu = b.take<double>(ny);
  double *kx2 = b.take<double>(mp), *kz2 = b.take<double>(nz);
  double *rowsN = b.take<double>(3 * (size_t)ny), *rowsD = b.take<double>(3 * (size_t)ny);
  double* cn = b.take<double>(9 * kCnKinds * (size_t)ny);
  void *twx = b.take<cplx<double>>(nx / 2), *twp = b.take<cplx<double>>(nx / 2 + 1), *twz = b.take<cplx<double>>(nz);
  void *twxf = b.take<cplx<float>>(nx / 2), *twpf = b.take<cplx<float>>(nx / 2 + 1), *twzf = b.take<cplx<float>>(nz);
  double* dpart = b.take<double>((size_t)kDiagBlocks * 16);
  double* dout = b.take<double>(16);
  int* st = b.take<int>(4);
  double* probe = b.take<double>((size_t)kProbeBlocks * 256);
  float *cpS = b.take<float>(nc), *cmS = b.take<float>(nc), *phiS = b.take<float>(nc);
  float *HcpS = b.take<float>(nc), *HcmS = b.take<float>(nc);
  float* mf[8];
  for (int q = 0; q < 8; ++q) mf[q] = b.take<float>(ny);
  float2* dgw = b.take<float2>(3 * (size_t)ny);
  float* cnF = b.take<float>(9 * kCnKinds * (size_t)ny);
  float *crefp = b.take<float>(ny), *crefm = b.take<float>(ny), *crfp = b.take<float>(ny), *crfm = b.take<float>(ny);
  float *rhoref = b.take<float>(ny), *rhorf = b.take<float>(ny), *dPref = b.take<float>(ny), *Fvref = b.take<float>(ny);
  double *Rrefp = b.take<double>(3 * (size_t)ny), *Rrefm = b.take<double>(3 * (size_t)ny);
  double *cr64p = b.take<double>(ny), *cr64m = b.take<double>(ny), *Pr64 = b.take<double>(ny);
  double *mrhs = b.take<double>(ny), *mshift = b.take<double>(ny), *delta = b.take<double>(ny);
  double *Hrp = b.take<double>(ny), *Hrm = b.take<double>(ny);
  double *fcN = b.take<double>(nspec), *fiN = b.take<double>(nspec), *fcD = b.take<double>(nspec),
         *fiD = b.take<double>(nspec);
  cplx<double>* dscr = b.take<cplx<double>>(nspec);
  void* spec2 = b.take<cplx<double>>(nspec);
  cplx<double>* dscr2 = b.take<cplx<double>>(nspec);
  const size_t P2 = 2 * (size_t)nz * nx;
  void* wallu = b.take<char>(P2 * tv);
  void* wallw = b.take<char>(P2 * tv);
  float* fX = b.take<float>(P2 * 5 * 8);
  float* fY = b.take<float>(P2 * 5);
  float* fYp = b.take<float>(P2 * 5);
  const bool mixed = precision == PNP_MIXED;
  float2 *sfcN = b.take<float2>(mixed ? nspec : 0), *sfiN = b.take<float2>(mixed ? nspec : 0);
  float2 *sfcD = b.take<float2>(mixed ? nspec : 0), *sfiD = b.take<float2>(mixed ? nspec : 0);
  float2 *sfaN = b.take<float2>(mixed ? ny : 0), *sfaD = b.take<float2>(mixed ? ny : 0);
  float *cpL = b.take<float>(mixed ? nc : 0), *cmL = b.take<float>(mixed ? nc : 0);
  float2 *dCp2 = b.take<float2>(3 * (size_t)ny), *dCm2 = b.take<float2>(3 * (size_t)ny);
  double *wB = b.take<double>((size_t)nz * nx), *wT = b.take<double>((size_t)nz * nx);
  double* lift64 = b.take<double>(nc);
  float* lift32 = b.take<float>(nc);
  double* sacc = b.take<double>(12 * (size_t)ny);
  float* fuseG = b.take<float>(3 * kCnKinds * (size_t)ny);
  double* afd = b.take<double>(36 * (size_t)(nx + nz));
  float* aff = b.take<float>(36 * (size_t)(nx + nz));
  if (c) {
    c->af_d = afd;
    c->af_f = aff;
    c->stats_acc = sacc;
    c->fuseG_d = fuseG;
    c->wallB_d = wB; c->wallT_d = wT; c->lift64 = lift64; c->lift32 = lift32;
    c->dCp_f2 = dCp2; c->dCm_f2 = dCm2;
    c->spf_cprN = sfcN; c->spf_invN = sfiN; c->spf_cprD = sfcD; c->spf_invD = sfiD;
    c->spf_aN = sfaN; c->spf_aD = sfaD;
    c->cpL = cpL; c->cmL = cmL;
    c->dscr = dscr;
    c->spec2 = spec2;
    c->dscr2 = dscr2;
    c->wall_u = wallu; c->wall_w = wallw; c->featX = fX; c->featY = fY; c->featYprev = fYp;
    c->spc_cprN = fcN; c->spc_invN = fiN; c->spc_cprD = fcD; c->spc_invD = fiD;
    c->cpS = cpS; c->cmS = cmS; c->phiS = phiS; c->HcpS = HcpS; c->HcmS = HcmS;
    for (int q = 0; q < 8; ++q) c->mf[q] = mf[q];
    c->diag_w = dgw;
    c->cnF_d = cnF;
    c->crefp_f = crefp; c->crefm_f = crefm; c->crfp_f = crfp; c->crfm_f = crfm;
    c->rhoref_f = rhoref; c->rhorf_f = rhorf; c->dPref_f = dPref; c->Fvref_f = Fvref;
    c->Rrefp_d = Rrefp; c->Rrefm_d = Rrefm; c->cref64p_d = cr64p; c->cref64m_d = cr64m; c->Phiref64_d = Pr64;
    c->meanrhs_d = mrhs; c->meanshift_d = mshift; c->delta_d = delta; c->Hrefp_d = Hrp; c->Hrefm_d = Hrm;
    c->u = u; c->v = v; c->w = w; c->p = p; c->Hu = Hu; c->Hv = Hv; c->Hw = Hw; c->ru = ru; c->rv = rv; c->rw = rw;
    c->cp = cp; c->cm = cm; c->Phi = Phi; c->Hcp = Hcp; c->Hcm = Hcm; c->rcp = rcp; c->rcm = rcm;
    c->sreal = sreal; c->spec = spec; c->stage = stage;
    c->yf_d = yf; c->yc_d = yc; c->idy_d = idy; c->ih_d = ih; c->lo_c_d = lo_c; c->hi_c_d = hi_c;
    c->lo_f_d = lo_f; c->hi_f_d = hi_f; c->wl_d = wl; c->wu_d = wu; c->kx2_d = kx2; c->kz2_d = kz2;
    c->rowsN_d = rowsN; c->rowsD_d = rowsD; c->cn_d = cn;
    c->twx_d = twx; c->twp_d = twp; c->twz_d = twz; c->twx_f = twxf; c->twp_f = twpf; c->twz_f = twzf;
    c->diag_partial = dpart; c->diag_out = dout; c->status_d = st; c->probe_d = probe;
    c->g.mh = mh;
    c->g.mp = mp;
    c->nc = nc;
    c->nv = nv;
  }
  return b.off + kAlign;
}

int check_grid(int nx, int ny, int nz) {
  if (!is_pow2(nx) || !is_pow2(nz) || nx < 4 || nz < 4 || nx > 4096 || nz > 4096 || ny < 3 || ny > 65536)
    return PNP_ERR_GRID;
  return PNP_OK;
}

#define CK(...)                                          \
  do {                                                   \
    if ((__VA_ARGS__) != cudaSuccess) return PNP_ERR_CUDA; \
  } while (0)

// Records the next site-boundary event when profiling or tracing (no-op
// otherwise): the end of site `site` (-1: a start) on stream st.
inline void mark(pnp_ctx* c, cudaStream_t st, int site) {
  if (c->prof && c->prof->n < Prof::kMax) {
    const int i = c->prof->n++;
    c->prof->site[i] = site;
    c->prof->on_aux[i] = st == c->aux;
    if (c->prof->external) cudaEventRecordWithFlags(c->prof->ev[i], st, cudaEventRecordExternal);
    else cudaEventRecord(c->prof->ev[i], st);
  }
}
// site timing or tracing with the concurrent schedule off
inline bool serial_sites(const pnp_ctx* c) { return c->prof && !c->prof->timeline; }

Metrics metrics(const pnp_ctx* c) {
  return Metrics{c->yc_d, c->idy_d, c->ih_d, c->lo_c_d, c->hi_c_d, c->lo_f_d, c->hi_f_d, c->wl_d, c->wu_d};
}

// Grid metrics and the y-operator rows (finite-volume forms of Fig. 1).
int upload_metrics(pnp_ctx* c) {
  const int ny = c->g.ny, nyc = c->g.nyc;
  std::vector<double>& yf = c->yf;
  yf[0] = -1.0;
  yf[ny - 1] = 1.0;
  c->yc.assign(nyc, 0.0);
  c->dy.assign(nyc, 0.0);
  c->h.assign(ny, 0.0);
  for (int j = 0; j < nyc; ++j) {
    c->dy[j] = yf[j + 1] - yf[j];
    c->yc[j] = 0.5 * (yf[j] + yf[j + 1]);
  }
  for (int j = 0; j < nyc; ++j)
    if (!(c->dy[j] > 0.0)) return PNP_ERR_GRID;
  c->h[0] = 0.5 * c->dy[0];
  for (int j = 1; j < nyc; ++j) c->h[j] = c->yc[j] - c->yc[j - 1];
  c->h[nyc] = 0.5 * c->dy[nyc - 1];
  std::vector<double> yc(ny, 0.0), idy(ny, 0.0), ih(ny, 0.0), loc(ny, 0.0), hic(ny, 0.0), lof(ny, 0.0),
      hif(ny, 0.0), wl(ny, 0.0), wu(ny, 0.0);
  for (int j = 0; j < nyc; ++j) {
    yc[j] = c->yc[j];
    idy[j] = 1.0 / c->dy[j];
    loc[j] = 1.0 / (c->h[j] * c->dy[j]);
    hic[j] = 1.0 / (c->h[j + 1] * c->dy[j]);
  }
  for (int j = 0; j < ny; ++j) ih[j] = 1.0 / c->h[j];
  for (int j = 1; j < nyc; ++j) {
    lof[j] = 1.0 / (c->dy[j - 1] * c->h[j]);
    hif[j] = 1.0 / (c->dy[j] * c->h[j]);
    wl[j] = c->dy[j - 1] / (2.0 * c->h[j]);
    wu[j] = c->dy[j] / (2.0 * c->h[j]);
  }
  // rows of d2/dy2 for cell-centred quantities (Neumann: zero wall flux; Dirichlet: wall value on the face)
  std::vector<double> rN(3 * (size_t)ny, 0.0), rD(3 * (size_t)ny, 0.0);
  for (int bc = 0; bc < 2; ++bc) {
    double* r = bc == 0 ? rN.data() : rD.data();
    double *a = r, *b = r + ny, *cc = r + 2 * ny;
    for (int j = 0; j < nyc; ++j) {
      const double lo = 1.0 / (c->h[j] * c->dy[j]);
      const double hi = 1.0 / (c->h[j + 1] * c->dy[j]);
      b[j] = 0.0;
      if (j > 0) { a[j] = lo; b[j] -= lo; }
      else if (bc == 1) b[j] -= lo;
      if (j < nyc - 1) { cc[j] = hi; b[j] -= hi; }
      else if (bc == 1) b[j] -= hi;
    }
  }
  const int nx = c->g.nx, nz = c->g.nz, mh = c->g.mh, mp = c->g.mp;
  std::vector<double> kx2(mp, 0.0), kz2(nz, 0.0);
  for (int m = 0; m < mh; ++m) kx2[m] = (2.0 - 2.0 * std::cos(2.0 * M_PI * m / nx)) / (c->g.dx * c->g.dx);
  for (int n = 0; n < nz; ++n) kz2[n] = (2.0 - 2.0 * std::cos(2.0 * M_PI * n / nz)) / (c->g.dz * c->g.dz);
  // FFT tables: exp(-2 pi i t / N)
  const int Lh = nx / 2;
  std::vector<cplx<double>> twx(Lh), twp(Lh + 1), twz(nz);
  std::vector<cplx<float>> twxf(Lh), twpf(Lh + 1), twzf(nz);
  for (int t = 0; t < Lh; ++t) twx[t] = {std::cos(2.0 * M_PI * t / Lh), -std::sin(2.0 * M_PI * t / Lh)};
  for (int t = 0; t <= Lh; ++t) twp[t] = {std::cos(2.0 * M_PI * t / nx), -std::sin(2.0 * M_PI * t / nx)};
  for (int t = 0; t < nz; ++t) twz[t] = {std::cos(2.0 * M_PI * t / nz), -std::sin(2.0 * M_PI * t / nz)};
  for (int t = 0; t < Lh; ++t) twxf[t] = {(float)twx[t].x, (float)twx[t].y};
  for (int t = 0; t <= Lh; ++t) twpf[t] = {(float)twp[t].x, (float)twp[t].y};
  for (int t = 0; t < nz; ++t) twzf[t] = {(float)twz[t].x, (float)twz[t].y};
  cudaStream_t s = c->stream;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
  };
  const size_t B = sizeof(double) * ny;
  CK(up(c->yf_d, yf.data(), B));
  CK(up(c->yc_d, yc.data(), B));
  CK(up(c->idy_d, idy.data(), B));
  CK(up(c->ih_d, ih.data(), B));
  CK(up(c->lo_c_d, loc.data(), B));
  CK(up(c->hi_c_d, hic.data(), B));
  CK(up(c->lo_f_d, lof.data(), B));
  CK(up(c->hi_f_d, hif.data(), B));
  CK(up(c->wl_d, wl.data(), B));
  CK(up(c->wu_d, wu.data(), B));
  CK(up(c->rowsN_d, rN.data(), 3 * B));
  CK(up(c->rowsD_d, rD.data(), 3 * B));
  CK(up(c->kx2_d, kx2.data(), sizeof(double) * mp));
  CK(up(c->kz2_d, kz2.data(), sizeof(double) * nz));
  CK(up(c->twx_d, twx.data(), sizeof(cplx<double>) * Lh));
  CK(up(c->twp_d, twp.data(), sizeof(cplx<double>) * (Lh + 1)));
  CK(up(c->twz_d, twz.data(), sizeof(cplx<double>) * nz));
  CK(up(c->twx_f, twxf.data(), sizeof(cplx<float>) * Lh));
  CK(up(c->twp_f, twpf.data(), sizeof(cplx<float>) * (Lh + 1)));
  CK(up(c->twz_f, twzf.data(), sizeof(cplx<float>) * nz));
  {
    const std::vector<double>* src[8] = {&idy, &ih, &loc, &hic, &lof, &hif, &wl, &wu};
    std::vector<float> tmp(8 * (size_t)ny);
    for (int q = 0; q < 8; ++q)
      for (int j = 0; j < ny; ++j) tmp[(size_t)q * ny + j] = (float)(*src[q])[j];
    for (int q = 0; q < 8; ++q) CK(up(c->mf[q], tmp.data() + (size_t)q * ny, sizeof(float) * ny));
    std::vector<float2> w(3 * (size_t)ny, make_float2(0.f, 0.f));
    auto split = [](double x) { return make_float2((float)x, (float)(x - (double)(float)x)); };
    for (int j = 0; j < nyc; ++j) w[j] = split(c->dy[j]);
    for (int j = 0; j < ny; ++j) w[ny + j] = split(c->h[j]);
    for (int j = 0; j < nyc; ++j) w[2 * (size_t)ny + j] = split(1.0 / c->dy[j]);
    CK(up(c->diag_w, w.data(), sizeof(float2) * 3 * ny));
    CK(cudaStreamSynchronize(s));
  }
  {
    const YRows rn{c->rowsN_d, c->rowsN_d + ny, c->rowsN_d + 2 * ny};
    const YRows rd{c->rowsD_d, c->rowsD_d + ny, c->rowsD_d + 2 * ny};
    CK(launch_spec_factors(c->spc_cprN, c->spc_invN, c->kx2_d, c->kz2_d, rn, c->g, true, s));
    CK(launch_spec_factors(c->spc_cprD, c->spc_invD, c->kx2_d, c->kz2_d, rd, c->g, false, s));
    if (c->precision == PNP_MIXED) {
      const size_t nspec = (size_t)c->g.nyc * c->g.nz * c->g.mp;
      CK(launch_to_df(c->spc_cprN, c->spf_cprN, nspec, s));
      CK(launch_to_df(c->spc_invN, c->spf_invN, nspec, s));
      CK(launch_to_df(c->spc_cprD, c->spf_cprD, nspec, s));
      CK(launch_to_df(c->spc_invD, c->spf_invD, nspec, s));
      CK(launch_to_df(c->rowsN_d, c->spf_aN, (size_t)ny, s));
      CK(launch_to_df(c->rowsD_d, c->spf_aD, (size_t)ny, s));
    }
  }
  CK(cudaStreamSynchronize(s));   // host vectors above are temporaries
  c->refs_valid = false;
  c->cn_dt = NAN;
  c->graph_dt = NAN;
  return PNP_OK;
}

// Elimination factors of (I - s L_y) for the three substages and three kinds
// (0: u and w, Dirichlet wall values on the faces; 1: v on interior faces;
// 2: ions, zero wall flux), s = alp dt nu / 2 (nu = 1/Re or 1/(Re Sc)).
int upload_cn(pnp_ctx* c, double dt) {
  const int ny = c->g.ny, nyc = c->g.nyc;
  c->cn_h.assign(9 * kCnKinds * (size_t)ny, 0.0);
  for (int l = 0; l < 3; ++l) {
    const double alp = kGam[l] + kZet[l];
    for (int kind = 0; kind < kCnKinds; ++kind) {
      const double diff = kind == 2 ? c->ph.D : c->ph.nu;
      const double sfac = 0.5 * alp * dt * diff;
      const int n = kind == 1 ? nyc - 1 : nyc;
      std::vector<double> a(n, 0.0), b(n, 0.0), cc(n, 0.0);
      for (int idx = 0; idx < n; ++idx) {
        if (kind == 1) {
          const int j = idx + 1;
          const double lo = 1.0 / (c->dy[j - 1] * c->h[j]);
          const double hi = 1.0 / (c->dy[j] * c->h[j]);
          if (idx > 0) a[idx] = lo;
          if (idx < n - 1) cc[idx] = hi;
          b[idx] = -lo - hi;
        } else {
          const int j = idx;
          const double lo = 1.0 / (c->h[j] * c->dy[j]);
          const double hi = 1.0 / (c->h[j + 1] * c->dy[j]);
          const bool dir = kind == 0;
          if (j > 0) { a[j] = lo; b[j] -= lo; }
          else if (dir) b[j] -= lo;
          if (j < nyc - 1) { cc[j] = hi; b[j] -= hi; }
          else if (dir) b[j] -= hi;
        }
      }
      double* A = c->cn_h.data() + ((size_t)(l * kCnKinds + kind) * 3 + 0) * ny;
      double* Cp = c->cn_h.data() + ((size_t)(l * kCnKinds + kind) * 3 + 1) * ny;
      double* M = c->cn_h.data() + ((size_t)(l * kCnKinds + kind) * 3 + 2) * ny;
      double cprev = 0.0;
      for (int idx = 0; idx < n; ++idx) {
        const double Aj = -sfac * a[idx], Bj = 1.0 - sfac * b[idx], Cj = -sfac * cc[idx];
        const double m = idx == 0 ? Bj : Bj - Aj * cprev;
        cprev = Cj / m;
        A[idx] = Aj;
        Cp[idx] = cprev;
        M[idx] = 1.0 / m;
      }
    }
  }
  std::vector<float> cnf(9 * kCnKinds * (size_t)ny, 0.f);
  for (size_t q = 0; q < cnf.size(); ++q) cnf[q] = (float)c->cn_h[q];
  CK(cudaMemcpyAsync(c->cn_d, c->cn_h.data(), sizeof(double) * c->cn_h.size(), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->cnF_d, cnf.data(), sizeof(float) * cnf.size(), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->cn_dt = dt;
  c->refs_dt = NAN;
  c->fuse_dt = NAN;
  c->af_dt = NAN;
  return PNP_OK;
}

// The stencil eliminates forward chunk by chunk (chunk length jc) when the
// mixed path runs its default policy with the line back substitution.
// The approximate factorisation fuses too: the y-elimination (chunk-local
// forward values, chunk carries, back substitution) is linear and the same for
// every (x, z) column, the x/z sweeps linear and the same for every y-plane, so
// the sweeps act on the stencil's forward values as they would on the
// right-hand sides, between the stencil and the back substitution.
bool cn_fused(const pnp_ctx* c, int* jc_out = nullptr) {
  if (c->precision != PNP_MIXED || c->policy != PNP_POLICY_DEFAULT || !c->fuse_cn || c->g.lc_cn == 32)
    return false;
  const int jc = mixed_rhs_chunk(c->g, c->rhs_maps_ok);
  if ((c->g.nyc - 1) / jc + 1 > kFusedMaxChunks) return false;
  if (jc_out) *jc_out = jc;
  return true;
}

// Chunk products G_r = prod_{i=s..r} (-a_i m_i) over the rows of each chunk,
// from the FP32 factor rows the stencil eliminates with (needs upload_cn's dt).
int upload_fuse(pnp_ctx* c, double dt, int jc) {
  const int ny = c->g.ny, nyc = c->g.nyc;
  std::vector<float> G(3 * kCnKinds * (size_t)ny, 0.f);
  for (int l = 0; l < 3; ++l)
    for (int kind = 0; kind < kCnKinds; ++kind) {
      const double* A = c->cn_h.data() + ((size_t)(l * kCnKinds + kind) * 3 + 0) * ny;
      const double* M = c->cn_h.data() + ((size_t)(l * kCnKinds + kind) * 3 + 2) * ny;
      const int n = kind == 1 ? nyc - 1 : nyc, j0 = kind == 1 ? 1 : 0;
      float* out = G.data() + (size_t)(l * kCnKinds + kind) * ny;
      double acc = 1.0;
      for (int r = 0; r < n; ++r) {
        if (r == 0 || (r + j0) % jc == 0) acc = 1.0;   // first row of a chunk
        acc *= -(double)(float)A[r] * (double)(float)M[r];
        out[r] = (float)acc;
      }
    }
  CK(cudaMemcpyAsync(c->fuseG_d, G.data(), sizeof(float) * G.size(), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->fuse_dt = dt;
  c->fuse_jc = jc;
  return PNP_OK;
}

// Offset (in values) of the periodic-sweep factors of (substage l, kind k, dir d).
size_t af_off(const pnp_ctx* c, int l, int k, int d) {
  const size_t nx = c->g.nx, nz = c->g.nz;
  return (size_t)(l * 2 + k) * 3 * (nx + nz) + (d ? 3 * nx : 0);
}

// Factors of the cyclic systems (I - s L) along x and z, s = alp dt nu / 2 or
// alp dt D / 2: diagonal 1 + 2 s / h^2, off-diagonals -s / h^2, wrapping.  The
// Thomas factors of the corner-free system with the two modified end
// diagonals, the Sherman-Morrison vector q = T^-1 (gam, 0, .., 0, up) and the
// scalars lo, lo / gam, 1 / (1 + q_0 + (lo / gam) q_{n-1}).
int upload_af(pnp_ctx* c, double dt) {
  const size_t tot = 36 * (size_t)(c->g.nx + c->g.nz);
  std::vector<double> h(tot, 0.0);
  for (int l = 0; l < 3; ++l) {
    const double alp = kGam[l] + kZet[l];
    for (int k = 0; k < 2; ++k) {
      const double s = 0.5 * alp * dt * (k == 0 ? c->ph.nu : c->ph.D);
      for (int d = 0; d < 2; ++d) {
        const int n = d ? c->g.nz : c->g.nx;
        const double hh = d ? c->g.dz : c->g.dx;
        const double beta = s / (hh * hh), lo = -beta, up = -beta, di = 1.0 + 2.0 * beta, gam = -di;
        double* cp = h.data() + af_off(c, l, k, d);
        double* m = cp + n;
        double* q = m + n;
        // forward factors of T (a = lo for i >= 1, b_0 = di - gam, b_{n-1} = di - lo up / gam)
        double cprev = 0.0;
        for (int i = 0; i < n; ++i) {
          const double b = i == 0 ? di - gam : (i == n - 1 ? di - lo * up / gam : di);
          const double piv = i == 0 ? b : b - lo * cprev;
          m[i] = 1.0 / piv;
          cprev = (i < n - 1 ? up : 0.0) * m[i];
          cp[i] = cprev;
        }
        // q = T^-1 u, u = (gam, 0, ..., 0, up)
        double dd = 0.0;
        std::vector<double> dv(n);
        for (int i = 0; i < n; ++i) {
          const double ui = i == 0 ? gam : (i == n - 1 ? up : 0.0);
          dd = (ui - (i ? lo * dd : 0.0)) * m[i];
          dv[i] = dd;
        }
        double y = dv[n - 1];
        q[n - 1] = y;
        for (int i = n - 2; i >= 0; --i) {
          y = dv[i] - cp[i] * y;
          q[i] = y;
        }
        c->af_sc[l][k][d][0] = lo;
        c->af_sc[l][k][d][1] = lo / gam;
        c->af_sc[l][k][d][2] = 1.0 / (1.0 + q[0] + (lo / gam) * q[n - 1]);
        // g = (I - s L)^-1 e_0 by the same cyclic solve (Thomas on the corner-free
        // system, back substitution, Sherman-Morrison correction)
        std::vector<double> gv(n);
        double d2 = 0.0;
        for (int i = 0; i < n; ++i) {
          d2 = ((i == 0 ? 1.0 : 0.0) - (i ? lo * d2 : 0.0)) * m[i];
          gv[i] = d2;
        }
        const double glast = gv[n - 1];
        for (int i = n - 2; i >= 0; --i) gv[i] -= cp[i] * gv[i + 1];
        const double fcor = (gv[0] + (lo / gam) * glast) * c->af_sc[l][k][d][2];
        for (int i = 0; i < n; ++i) gv[i] -= fcor * q[i];
        double tot = 0.0;
        for (int i = 0; i < n; ++i) tot += std::fabs(gv[i]);
        for (int t = 0; t <= kConvMaxK; ++t)   // symmetric: g_t = g_(n-t)
          c->af_g[l][k][d][t] = 2 * t < n ? 0.5 * (gv[t] + gv[(n - t) % n]) : 0.0;
        // taps past which the dropped tail sum_(K < t < n - K) |g_t| is below the
        // pass's rounding (2^-27 of sum |g| for FP32, 2^-54 for FP64)
        auto taps = [&](double rel) {
          for (int K = 0; K <= kConvMaxK && 2 * K + 1 <= n; ++K) {
            double tail = 0.0;
            for (int t = K + 1; t < n - K; ++t) tail += std::fabs(gv[t]);
            if (tail <= rel * tot) return K;
          }
          return -1;
        };
        c->af_kf[l][k][d] = taps(std::ldexp(1.0, -27));
        c->af_kd[l][k][d] = taps(std::ldexp(1.0, -54));
      }
    }
  }
  std::vector<float> f(tot);
  for (size_t q = 0; q < tot; ++q) f[q] = (float)h[q];
  CK(cudaMemcpyAsync(c->af_d, h.data(), sizeof(double) * tot, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->af_f, f.data(), sizeof(float) * tot, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->af_dt = dt;
  return PNP_OK;
}

// Periodic sweeps (x, then z) of the approximate factorisation on the CN
// right-hand sides of substage l: families u, v (interior faces), w (fam bit 1)
// and c+, c- (fam bit 2), in the context's precision.
template <typename TR>
cudaError_t periodic_sweeps(pnp_ctx* c, int l, unsigned fams, TR* ru, TR* rv, TR* rw, TR* rcp, TR* rcm,
                            cudaStream_t st) {
  const size_t P = (size_t)c->g.nz * c->g.nx;
  // one pass of truncated convolutions when every family's taps fit
  // (the launch's shapes: 16-byte vectors of columns, at most 512 per row; x
  // taps rounded up to 4 or 8, z taps to 2, 4 or 8, each within half a line)
  auto ktaps = [&](int k, int d) { return sizeof(TR) == 8 ? c->af_kd[l][k][d] : c->af_kf[l][k][d]; };
  const int vec = 16 / (int)sizeof(TR);
  bool conv = c->g.nx % vec == 0 && c->g.nx / vec <= 512;
  int kx = 0, kz = 2;
  for (int k = 0; k < 2; ++k)
    if (fams & (1u << k)) {
      if (ktaps(k, 0) < 0 || ktaps(k, 1) < 0) conv = false;
      kx = std::max(kx, ktaps(k, 0));
      kz = std::max(kz, ktaps(k, 1));
    }
  int kzr = 2;
  while (kzr < kz) kzr <<= 1;
  const int kxr = kx <= 4 ? 4 : 8;
  if (conv && kzr <= kConvMaxK && 2 * kzr + 1 <= c->g.nz && kx <= kConvMaxK && 2 * kxr + 1 <= c->g.nx) {
    ConvArgs<TR> a{};
    a.kz = kzr;
    auto fam = [&](TR* r, int np, int k) {
      ConvFam<TR> F{};
      F.r = r;
      F.nplanes = np;
      F.kx = ktaps(k, 0);
      for (int t = 0; t <= kConvMaxK; ++t) {
        F.gx[t] = t <= kxr ? (TR)c->af_g[l][k][0][t] : TR(0);
        F.gz[t] = t <= kzr ? (TR)c->af_g[l][k][1][t] : TR(0);
      }
      a.f[a.nfam++] = F;
    };
    if (fams & 1u) {
      fam(ru, c->g.nyc, 0);
      fam(rv + P, c->g.nyc - 1, 0);
      fam(rw, c->g.nyc, 0);
    }
    if (fams & 2u) {
      fam(rcp, c->g.nyc, 1);
      fam(rcm, c->g.nyc, 1);
    }
    return launch_periodic_conv<TR>(a, c->g, st);
  }
  for (int d = 0; d < 2; ++d) {
    PeriodicArgs<TR> a{};
    auto fam = [&](TR* r, int np, int k) {
      const int n = d ? c->g.nz : c->g.nx;
      const size_t off = af_off(c, l, k, d);
      const TR* base = sizeof(TR) == 8 ? (const TR*)(c->af_d + off) : (const TR*)(c->af_f + off);
      a.f[a.nfam++] = PeriodicFam<TR>{r, np, base, base + n, base + 2 * n, (TR)c->af_sc[l][k][d][0],
                                      (TR)c->af_sc[l][k][d][1], (TR)c->af_sc[l][k][d][2]};
    };
    if (fams & 1u) {
      fam(ru, c->g.nyc, 0);
      fam(rv + P, c->g.nyc - 1, 0);
      fam(rw, c->g.nyc, 0);
    }
    if (fams & 2u) {
      fam(rcp, c->g.nyc, 1);
      fam(rcm, c->g.nyc, 1);
    }
    const cudaError_t e = launch_periodic<TR>(a, c->g, d == 1, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The factor tables a step of size dt needs (CN rows, fused-chunk products,
// periodic-sweep factors).
int prepare_tables(pnp_ctx* c, double dt) {
  if (c->cn_dt != dt) {
    int r = upload_cn(c, dt);
    if (r) return r;
  }
  if (c->scheme == PNP_SCHEME_AF && !(c->af_dt == dt)) {
    int r = upload_af(c, dt);
    if (r) return r;
  }
  int jc = 0;
  if (cn_fused(c, &jc) && (!(c->fuse_dt == dt) || c->fuse_jc != jc)) return upload_fuse(c, dt, jc);
  return PNP_OK;
}

CNRows cn_rows(const pnp_ctx* c, int l, int kind) {
  const size_t ny = c->g.ny;
  const double* base = c->cn_d + (size_t)(l * kCnKinds + kind) * 3 * ny;
  return CNRows{base, base + ny, base + 2 * ny};
}

CNRowsF cn_rows_f(const pnp_ctx* c, int l, int kind) {
  const size_t ny = c->g.ny;
  const float* base = c->cnF_d + (size_t)(l * kCnKinds + kind) * 3 * ny;
  return CNRowsF{base, base + ny, base + 2 * ny};
}

MetricsF metrics_f(const pnp_ctx* c) {
  return MetricsF{c->mf[0], c->mf[1], c->mf[2], c->mf[3], c->mf[4], c->mf[5], c->mf[6], c->mf[7]};
}

CoefF coef_f(const pnp_ctx* c, const Stage& st, bool keep_h = true) {
  CoefF f{(float)c->g.idx, (float)c->g.idz, (float)c->ph.nu, (float)c->ph.D, (float)c->ph.K, (float)c->ph.Uw,
          (float)st.dt, (float)st.gam, (float)st.zet, (float)st.alp};
  f.idx2 = f.idx * f.idx;
  f.idz2 = f.idz * f.idz;
  f.Kx = f.K * f.idx;
  f.Kz = f.K * f.idz;
  f.Dx = f.D * f.idx;
  f.Dz = f.D * f.idz;
  f.anu = f.alp * f.nu;
  f.aD = f.alp * f.D;
  f.keep_h = keep_h ? 1 : 0;
  f.af = st.af;
  f.nuH = st.af ? 0.f : f.nu;
  f.anuxz = st.af ? (float)(st.alp * c->ph.nu) : 0.f;
  f.zD = st.af ? (float)(st.zet * c->ph.D) : 0.f;
  return f;
}

const RhsMaps* rhs_maps(const pnp_ctx* c) { return c->rhs_maps_ok ? &c->rhs_maps : nullptr; }

Shadows shadows(const pnp_ctx* c) { return Shadows{c->cpS, c->cmS, c->phiS, c->HcpS, c->HcmS, c->cpL, c->cmL}; }

MixedRefs mixed_refs(const pnp_ctx* c) {
  return MixedRefs{c->crefp_f, c->crefm_f, c->crfp_f, c->crfm_f, c->rhoref_f, c->rhorf_f, c->dPref_f, c->Fvref_f,
                   c->Rrefp_d, c->Rrefm_d, c->cref64p_d, c->cref64m_d, c->Phiref64_d, c->meanrhs_d,
                   c->meanshift_d, c->delta_d, c->dCp_f2, c->dCm_f2};
}

SpecDF spec_df(const pnp_ctx* c, bool neumann) {
  return neumann ? SpecDF{c->spf_cprN, c->spf_invN, c->spf_aN} : SpecDF{c->spf_cprD, c->spf_invD, c->spf_aD};
}

YRows yrows(const pnp_ctx* c, bool neumann) {
  const double* r = neumann ? c->rowsN_d : c->rowsD_d;
  const size_t ny = c->g.ny;
  return YRows{r, r + ny, r + 2 * ny};
}

template <typename TV>
Fields<TV> fields(const pnp_ctx* c) {
  Fields<TV> f;
  f.u = (TV*)c->u; f.v = (TV*)c->v; f.w = (TV*)c->w; f.p = (TV*)c->p;
  f.Hu = (TV*)c->Hu; f.Hv = (TV*)c->Hv; f.Hw = (TV*)c->Hw;
  f.ru = (TV*)c->ru; f.rv = (TV*)c->rv; f.rw = (TV*)c->rw;
  f.cp = c->cp; f.cm = c->cm; f.Phi = c->Phi; f.Hcp = c->Hcp; f.Hcm = c->Hcm; f.rcp = c->rcp; f.rcm = c->rcm;
  f.wall_u = c->slip_on ? (const TV*)c->wall_u : nullptr;
  f.wall_w = c->slip_on ? (const TV*)c->wall_w : nullptr;
  return f;
}

// Spectral part of a separable Poisson solve: z-FFT, Thomas per (m, n), inverse z-FFT.
template <typename T>
cudaError_t spectral_solve(pnp_ctx* c, cplx<T>* spec, const cplx<T>* twz, bool neumann, cudaStream_t st,
                           cplx<double>* dscr) {
  cudaError_t e = launch_fft_z<T>(spec, twz, c->g, false, st);
  if (e != cudaSuccess) return e;
  mark(c, st, neumann ? PNP_SITE_P_FFTZ : PNP_SITE_E_FFTZ);
  const double scale = 1.0 / ((double)c->g.nx * (double)c->g.nz);
  if constexpr (sizeof(T) == sizeof(float))
    e = launch_spec_thomas_df(spec, dscr, spec_df(c, neumann), neumann ? c->spc_cprN : c->spc_cprD,
                              neumann ? c->spc_invN : c->spc_invD, yrows(c, neumann), c->g, scale, neumann, st);
  else
    e = launch_spec_thomas<T>(spec, dscr, neumann ? c->spc_cprN : c->spc_cprD, neumann ? c->spc_invN : c->spc_invD,
                              yrows(c, neumann), c->g, scale, neumann, st);
  if (e != cudaSuccess) return e;
  mark(c, st, neumann ? PNP_SITE_P_THOMAS : PNP_SITE_E_THOMAS);
  e = launch_fft_z<T>(spec, twz, c->g, true, st);
  mark(c, st, neumann ? PNP_SITE_P_IFFTZ : PNP_SITE_E_IFFTZ);
  return e;
}

template <typename T>
cudaError_t spectral_solve(pnp_ctx* c, cplx<T>* spec, const cplx<T>* twz, bool neumann) {
  return spectral_solve<T>(c, spec, twz, neumann, c->stream, c->dscr);
}

// Pressure correction (Neumann) from div(u_hat) / scale and the projection.
template <typename TV>
cudaError_t pressure_projection(pnp_ctx* c, double scale, bool update_p) {
  const Metrics m = metrics(c);
  const Fields<TV> f = fields<TV>(c);
  cplx<TV>* spec = (cplx<TV>*)c->spec;
  const cplx<TV>* twx = (const cplx<TV>*)(sizeof(TV) == 8 ? c->twx_d : c->twx_f);
  const cplx<TV>* twp = (const cplx<TV>*)(sizeof(TV) == 8 ? c->twp_d : c->twp_f);
  const cplx<TV>* twz = (const cplx<TV>*)(sizeof(TV) == 8 ? c->twz_d : c->twz_f);
  TV* phip = (TV*)c->sreal;
  const TV* idyT = (const TV*)(sizeof(TV) == 8 ? (const void*)c->idy_d : (const void*)c->mf[0]);
  cudaError_t e = launch_fft_x_fwd<TV, TV>(PoissonSrc::Divergence, f.u, f.v, f.w, nullptr, nullptr, nullptr,
                                           1.0 / scale, c->g, m, spec, twx, twp, c->stream, nullptr, nullptr, idyT);
  if (e != cudaSuccess) return e;
  mark(c, c->stream, PNP_SITE_P_FFTX);
  e = spectral_solve<TV>(c, spec, twz, true);
  if (e != cudaSuccess) return e;
  e = launch_fft_x_inv<TV, TV>(PoissonDst::Plain, spec, c->g, m, twx, twp, 0.0, phip, c->stream);
  if (e != cudaSuccess) return e;
  mark(c, c->stream, PNP_SITE_P_IFFTX);
  const TV* ihT = (const TV*)(sizeof(TV) == 8 ? (const void*)c->ih_d : (const void*)c->mf[1]);
  e = launch_project<TV>(f.u, f.v, f.w, f.p, phip, scale, update_p, c->g, ihT, c->stream);
  mark(c, c->stream, PNP_SITE_PROJECT);
  return e;
}

// Eq. (4): L phi = -(c+ - c-) / (2 lam^2), phi = 0 on the walls; Phi = V y + phi (FP64).
template <typename TV>
cudaError_t potential_solve(pnp_ctx* c, cudaStream_t st, void* spec_buf, cplx<double>* dscr) {
  const Metrics m = metrics(c);
  cplx<double>* spec = (cplx<double>*)spec_buf;
  const cplx<double>* twx = (const cplx<double>*)c->twx_d;
  const cplx<double>* twp = (const cplx<double>*)c->twp_d;
  const cplx<double>* twz = (const cplx<double>*)c->twz_d;
  cudaError_t e = launch_fft_x_fwd<double, TV>(PoissonSrc::Charge, nullptr, nullptr, nullptr, c->cp, c->cm, nullptr,
                                               c->ph.q, c->g, m, spec, twx, twp, st);
  if (e != cudaSuccess) return e;
  mark(c, st, PNP_SITE_E_FFTX);
  e = spectral_solve<double>(c, spec, twz, false, st, dscr);
  if (e != cudaSuccess) return e;
  e = launch_fft_x_inv<double, double>(PoissonDst::Potential, spec, c->g, m, twx, twp, c->ph.V, c->Phi, st, nullptr,
                                       c->wall_map ? c->lift64 : nullptr);
  mark(c, st, PNP_SITE_E_IFFTX);
  return e;
}

template <typename TV>
cudaError_t potential_solve(pnp_ctx* c) {
  return potential_solve<TV>(c, c->stream, c->spec, c->dscr);
}

// Mixed potential: FP32 FFT of the fluctuating charge, FP64 y-solves and (0,0) mode.
cudaError_t potential_mixed(pnp_ctx* c, cudaStream_t st, void* spec_buf, cplx<double>* dscr) {
  const Shadows sh = shadows(c);
  const Metrics m = metrics(c);
  cplx<float>* spec = (cplx<float>*)spec_buf;
  const cplx<float>* twx = (const cplx<float>*)c->twx_f;
  const cplx<float>* twp = (const cplx<float>*)c->twp_f;
  const cplx<float>* twz = (const cplx<float>*)c->twz_f;
  cudaError_t e = launch_fft_x_fwd<float, float>(PoissonSrc::ChargeShadow, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                 nullptr, c->ph.q, c->g, m, spec, twx, twp, st, sh.cp, sh.cm);
  if (e != cudaSuccess) return e;
  mark(c, st, PNP_SITE_E_FFTX);
  e = launch_fft_z<float>(spec, twz, c->g, false, st);
  if (e != cudaSuccess) return e;
  mark(c, st, PNP_SITE_E_FFTZ);
  const double scale = 1.0 / ((double)c->g.nx * (double)c->g.nz);
  e = launch_spec_thomas_df(spec, dscr, spec_df(c, false), c->spc_cprD, c->spc_invD, yrows(c, false), c->g, scale,
                            false, st, c->meanrhs_d, c->meanshift_d, c->delta_d);
  if (e != cudaSuccess) return e;
  mark(c, st, PNP_SITE_E_THOMAS);
  e = launch_fft_z<float>(spec, twz, c->g, true, st);
  if (e != cudaSuccess) return e;
  mark(c, st, PNP_SITE_E_IFFTZ);
  e = launch_fft_x_inv<float, float>(PoissonDst::PotentialShadow, spec, c->g, m, twx, twp, 0.0, sh.phi, st, c->delta_d,
                                     c->wall_map ? c->lift32 : nullptr);
  mark(c, st, PNP_SITE_E_IFFTX);
  return e;
}

// The "FP64 solves" policy of the mixed path: both Poisson problems with FP64
// transforms, FP64 spectral y-solves and an FP64 (0,0) mode, from the FP32
// velocities and the double-float ion state; Phi_p and phi' stored in FP32.
cudaError_t pressure_projection_fp64(pnp_ctx* c, double scale) {
  const Metrics m = metrics(c);
  const Fields<float> f = fields<float>(c);
  cplx<double>* spec = (cplx<double>*)c->spec;
  const cplx<double>* twx = (const cplx<double>*)c->twx_d;
  const cplx<double>* twp = (const cplx<double>*)c->twp_d;
  const cplx<double>* twz = (const cplx<double>*)c->twz_d;
  float* phip = (float*)c->sreal;
  cudaError_t e = launch_fft_x_fwd<double, float>(PoissonSrc::Divergence, f.u, f.v, f.w, nullptr, nullptr, nullptr,
                                                  1.0 / scale, c->g, m, spec, twx, twp, c->stream, nullptr, nullptr,
                                                  c->idy_d);
  if (e != cudaSuccess) return e;
  mark(c, c->stream, PNP_SITE_P_FFTX);
  e = spectral_solve<double>(c, spec, twz, true, c->stream, c->dscr);
  if (e != cudaSuccess) return e;
  e = launch_fft_x_inv<double, float>(PoissonDst::Plain, spec, c->g, m, twx, twp, 0.0, phip, c->stream);
  if (e != cudaSuccess) return e;
  mark(c, c->stream, PNP_SITE_P_IFFTX);
  e = launch_project<float>(f.u, f.v, f.w, f.p, phip, scale, true, c->g, c->mf[1], c->stream);
  mark(c, c->stream, PNP_SITE_PROJECT);
  return e;
}

cudaError_t potential_mixed_fp64(pnp_ctx* c, cudaStream_t st, void* spec_buf, cplx<double>* dscr) {
  const Shadows sh = shadows(c);
  const Metrics m = metrics(c);
  cplx<double>* spec = (cplx<double>*)spec_buf;
  const cplx<double>* twx = (const cplx<double>*)c->twx_d;
  const cplx<double>* twp = (const cplx<double>*)c->twp_d;
  const cplx<double>* twz = (const cplx<double>*)c->twz_d;
  cudaError_t e = launch_fft_x_fwd<double, float>(PoissonSrc::ChargeShadowDF, nullptr, nullptr, nullptr, nullptr,
                                                  nullptr, nullptr, c->ph.q, c->g, m, spec, twx, twp, st, sh.cp,
                                                  sh.cm, nullptr, sh.cpL, sh.cmL);
  if (e != cudaSuccess) return e;
  mark(c, st, PNP_SITE_E_FFTX);
  e = launch_fft_z<double>(spec, twz, c->g, false, st);
  if (e != cudaSuccess) return e;
  mark(c, st, PNP_SITE_E_FFTZ);
  const double scale = 1.0 / ((double)c->g.nx * (double)c->g.nz);
  e = launch_spec_thomas<double>(spec, dscr, c->spc_cprD, c->spc_invD, yrows(c, false), c->g, scale, false, st,
                                 c->meanrhs_d, c->meanshift_d, c->delta_d);
  if (e != cudaSuccess) return e;
  mark(c, st, PNP_SITE_E_THOMAS);
  e = launch_fft_z<double>(spec, twz, c->g, true, st);
  if (e != cudaSuccess) return e;
  mark(c, st, PNP_SITE_E_IFFTZ);
  e = launch_fft_x_inv<double, float>(PoissonDst::PotentialShadow, spec, c->g, m, twx, twp, 0.0, sh.phi, st,
                                      c->delta_d, c->wall_map ? c->lift32 : nullptr);
  mark(c, st, PNP_SITE_E_IFFTX);
  return e;
}

// FP64 scratch of the FP64-arithmetic CN solves: the FP64 copies of the ion
// state, Phi, H_c+- and the conversion stage are not read during a mixed step
// (they are materialised on demand afterwards), so they hold the forward values.
CnScratch64 cn_scratch64(const pnp_ctx* c) {
  return CnScratch64{c->cp, c->stage, c->cm, c->Phi, c->Hcp};
}

// Pressure projection on the main stream and the potential solve, which
// depends only on the ions of this substage, on the auxiliary stream; joined
// before the substage ends.  Sequential when profiling (site timing).
template <typename TV>
cudaError_t poisson_pair(pnp_ctx* c, double scale) {
  auto pot = [&](cudaStream_t st, void* spec, cplx<double>* dscr) {
    return c->precision == PNP_FP64 ? potential_solve<TV>(c, st, spec, dscr) : potential_mixed(c, st, spec, dscr);
  };
  if (serial_sites(c)) {
    cudaError_t e = pressure_projection<TV>(c, scale, true);
    if (e != cudaSuccess) return e;
    return pot(c->stream, c->spec, c->dscr);
  }
  cudaError_t e = cudaEventRecord(c->ev_fork, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->aux, c->ev_fork, 0);
  if (e == cudaSuccess) e = pot(c->aux, c->spec2, c->dscr2);
  if (e == cudaSuccess) e = pressure_projection<TV>(c, scale, true);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->aux);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_join, 0);
  return e;
}



template <typename TV>
cudaError_t substage(pnp_ctx* c, double dt, int l) {
  const Stage st{dt, kGam[l], kZet[l], kGam[l] + kZet[l], c->scheme == PNP_SCHEME_AF ? 1 : 0};
  const Fields<TV> f = fields<TV>(c);
  mark(c, c->stream, -1);
  cudaError_t e = launch_rhs<TV>(f, c->g, metrics(c), c->ph, st, c->stream);
  if (e != cudaSuccess) return e;
  if (st.af) {
    e = periodic_sweeps<double>(c, l, 3u, (double*)f.ru, (double*)f.rv, (double*)f.rw, f.rcp, f.rcm, c->stream);
    if (e != cudaSuccess) return e;
  }
  mark(c, c->stream, PNP_SITE_RHS);
  e = launch_cn_solves<TV>(f, c->g, cn_rows(c, l, c->wall_stress ? 3 : 0), cn_rows(c, l, 1), cn_rows(c, l, 2),
                           c->stream);
  if (e != cudaSuccess) return e;
  mark(c, c->stream, PNP_SITE_CN);
  return poisson_pair<TV>(c, st.alp * dt);
}

// Mixed-precision substage (policy in k_mixed.cu).
cudaError_t substage_mixed(pnp_ctx* c, double dt, int l) {
  const Stage st{dt, kGam[l], kZet[l], kGam[l] + kZet[l], c->scheme == PNP_SCHEME_AF ? 1 : 0};
  const Fields<float> f = fields<float>(c);
  const Shadows sh = shadows(c);
  const MixedRefs R = mixed_refs(c);
  const bool fp64 = c->policy == PNP_POLICY_FP64_SOLVES;
  const int kc = c->wall_stress ? 3 : 0;   // u, w rows: Dirichlet wall values, or the wall-stress coupling
  const CNRowsF cell = cn_rows_f(c, l, kc), face = cn_rows_f(c, l, 1), ion = cn_rows_f(c, l, 2);
  int jc = 0;
  const bool fused = cn_fused(c, &jc) && c->fuse_dt == dt && c->fuse_jc == jc;
  const CnFuse fz{cell, face, ion, jc, fused ? 1 : 0};
  mark(c, c->stream, -1);
  cudaError_t e = launch_mixed_rhs(f, sh, R, c->g, metrics_f(c), coef_f(c, st, l < 2), rhs_maps(c), c->status_d + 1,
                                   c->stream, fused ? &fz : nullptr);
  if (e != cudaSuccess) return e;
  mark(c, c->stream, PNP_SITE_RHS);
  const size_t ny = c->g.ny;
  const float* Gl = c->fuseG_d + (size_t)l * kCnKinds * ny;
  const CnFusedG G{Gl + (size_t)kc * ny, Gl + ny, Gl + 2 * ny};
  auto cn = [&](unsigned parts, cudaStream_t s) {
    if (st.af) {   // the x/z factors first, on these families' FP32 right-hand sides (fused: forward values)
      const cudaError_t ea = periodic_sweeps<float>(c, l, (parts & kCnVelocity ? 1u : 0u) | (parts & kCnIons ? 2u : 0u),
                                                    f.ru, f.rv, f.rw, (float*)f.rcp, (float*)f.rcm, s);
      if (ea != cudaSuccess) return ea;
    }
    if (fp64)
      return launch_mixed_cn_fp64(f, sh, R, c->g, cn_rows(c, l, kc), cn_rows(c, l, 1), cn_rows(c, l, 2), l, parts,
                                  cn_scratch64(c), s);
    if (fused) return launch_mixed_cn_fused(f, sh, R, c->g, cell, face, ion, G, jc, l, parts, s);
    return launch_mixed_cn(f, sh, R, c->g, cell, face, ion, l, parts, s);
  };
  auto pot = [&](cudaStream_t s, void* spec, cplx<double>* dscr) {
    return fp64 ? potential_mixed_fp64(c, s, spec, dscr) : potential_mixed(c, s, spec, dscr);
  };
  auto proj = [&]() {
    return fp64 ? pressure_projection_fp64(c, st.alp * dt) : pressure_projection<float>(c, st.alp * dt, true);
  };
  if (serial_sites(c)) {   // site timing: everything in order on the main stream
    e = cn(kCnIons | kCnVelocity, c->stream);
    if (e != cudaSuccess) return e;
    mark(c, c->stream, PNP_SITE_CN);
    e = proj();
    if (e != cudaSuccess) return e;
    return pot(c->stream, c->spec, c->dscr);
  }
  // The ion CN solve and the potential depend only on the ions: both fork onto
  // the auxiliary stream right after the stencil and overlap the velocity CN
  // solve, the pressure pipeline and the projection.
  e = cudaEventRecord(c->ev_fork, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->aux, c->ev_fork, 0);
  if (e == cudaSuccess) e = cn(kCnIons, c->aux);
  if (e == cudaSuccess) mark(c, c->aux, PNP_SITE_CN);
  if (e == cudaSuccess) e = pot(c->aux, c->spec2, c->dscr2);
  if (e == cudaSuccess) e = cn(kCnVelocity, c->stream);
  if (e == cudaSuccess) mark(c, c->stream, PNP_SITE_CN);
  if (e == cudaSuccess) e = proj();
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->aux);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_join, 0);
  return e;
}

cudaError_t one_step(pnp_ctx* c, double dt) {
  for (int l = 0; l < 3; ++l) {
    cudaError_t e = c->precision == PNP_FP64 ? substage<double>(c, dt, l) : substage_mixed(c, dt, l);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void drop_graph(pnp_ctx* c);

// Mixed precision: bring the FP64 Phi and Hc+- arrays up to date from the shadows.
int materialize(pnp_ctx* c) {
  if (c->precision != PNP_MIXED || c->fp64_fresh) return PNP_OK;
  const size_t P = (size_t)c->g.nz * c->g.nx;
  CK(launch_from_shadow_df(c->cpS, c->cpL, c->cref64p_d, c->cp, P, c->nc, c->stream));
  CK(launch_from_shadow_df(c->cmS, c->cmL, c->cref64m_d, c->cm, P, c->nc, c->stream));
  CK(launch_from_shadow(c->phiS, c->Phiref64_d, c->Phi, P, c->nc, c->stream));
  CK(launch_from_shadow(c->HcpS, c->Hrefp_d, c->Hcp, P, c->nc, c->stream));
  CK(launch_from_shadow(c->HcmS, c->Hrefm_d, c->Hcm, P, c->nc, c->stream));
  c->fp64_fresh = true;
  return PNP_OK;
}

// c+, c-, Phi as the wall kernels read them: the shadows of a mixed context
// whose references are valid (what it steps on), else the FP64 arrays
// (brought up to date first).
int ion_view(pnp_ctx* c, IonView* v) {
  if (c->precision == PNP_MIXED && c->refs_valid) {
    *v = IonView{nullptr, nullptr, nullptr, c->cpS, c->cpL, c->cmS, c->cmL, c->phiS, c->cref64p_d, c->cref64m_d,
                 c->Phiref64_d};
    return PNP_OK;
  }
  int r = materialize(c);
  if (r) return r;
  *v = IonView{c->cp, c->cm, c->Phi, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  return PNP_OK;
}

// Mixed precision: reference profiles (plane means of c+, c-, Phi) and every
// per-plane FP64 constant derived from them; then the FP32 shadows.
int refresh_refs(pnp_ctx* c, double dt) {
  if (c->precision != PNP_MIXED) return PNP_OK;
  const int ny = c->g.ny, nyc = c->g.nyc;
  const size_t P = (size_t)c->g.nz * c->g.nx;
  if (!c->refs_valid) {
    int r = materialize(c);
    if (r) return r;
    CK(launch_plane_means3(c->cp, c->cm, c->Phi, nyc, P, c->cref64p_d, c->cref64m_d, c->Phiref64_d, c->stream));
    std::vector<double> cp(nyc), cm(nyc), Ph(nyc);
    CK(cudaMemcpyAsync(cp.data(), c->cref64p_d, sizeof(double) * nyc, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(cm.data(), c->cref64m_d, sizeof(double) * nyc, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(Ph.data(), c->Phiref64_d, sizeof(double) * nyc, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->refN_p = c->refN_m = 0.0;
    for (int j = 0; j < nyc; ++j) {
      c->refN_p += (double)P * cp[j] * c->dy[j];
      c->refN_m += (double)P * cm[j] * c->dy[j];
    }
    const double D = c->ph.D, K = c->ph.K, q = c->ph.q, V = c->ph.V;
    std::vector<float> crefp(ny, 0.f), crefm(ny, 0.f), crfp(ny, 0.f), crfm(ny, 0.f), rhoref(ny, 0.f), rhorf(ny, 0.f),
        dPref(ny, 0.f), Fvref(ny, 0.f);
    std::vector<double> mrhs(ny, 0.0), mshift(ny, 0.0);
    c->href_p.assign(ny, 0.0);
    c->href_m.assign(ny, 0.0);
    c->lyc_p.assign(ny, 0.0);
    c->lyc_m.assign(ny, 0.0);
    for (int j = 0; j < nyc; ++j) {
      crefp[j] = (float)cp[j];
      crefm[j] = (float)cm[j];
      rhoref[j] = (float)(cp[j] - cm[j]);
      mrhs[j] = -q * (cp[j] - cm[j]);
      mshift[j] = V * c->yc[j] + (c->wall_map ? c->wall_off : 0.0) - Ph[j];
    }
    // reference migration flux on interior faces, its divergence, the implicit
    // diffusion of the reference and the reference Coulomb force on v (all FP64)
    std::vector<double> Fp(ny, 0.0), Fm(ny, 0.0);
    for (int j = 1; j < nyc; ++j) {
      const double ih = 1.0 / c->h[j];
      const double dP = Ph[j] - Ph[j - 1];
      const double cfp = 0.5 * (cp[j - 1] + cp[j]), cfm = 0.5 * (cm[j - 1] + cm[j]);
      const double rf = 0.5 * ((cp[j - 1] - cm[j - 1]) + (cp[j] - cm[j]));
      Fp[j] = -1.0 * D * cfp * dP * ih;
      Fm[j] = +1.0 * D * cfm * dP * ih;
      crfp[j] = (float)cfp;
      crfm[j] = (float)cfm;
      rhorf[j] = (float)rf;
      dPref[j] = (float)dP;
      Fvref[j] = (float)(-K * rf * dP * ih);
    }
    c->refH_p = c->refH_m = 0.0;
    for (int j = 0; j < nyc; ++j) {
      const double idy = 1.0 / c->dy[j];
      c->href_p[j] = -(Fp[j + 1] - Fp[j]) * idy;
      c->href_m[j] = -(Fm[j + 1] - Fm[j]) * idy;
      c->refH_p += (double)P * c->href_p[j] * c->dy[j];
      c->refH_m += (double)P * c->href_m[j] * c->dy[j];
      const double lo = 1.0 / (c->h[j] * c->dy[j]), hi = 1.0 / (c->h[j + 1] * c->dy[j]);
      c->lyc_p[j] = (j > 0 ? lo * (cp[j - 1] - cp[j]) : 0.0) + (j < nyc - 1 ? hi * (cp[j + 1] - cp[j]) : 0.0);
      c->lyc_m[j] = (j > 0 ? lo * (cm[j - 1] - cm[j]) : 0.0) + (j < nyc - 1 ? hi * (cm[j + 1] - cm[j]) : 0.0);
    }
    auto upf = [&](float* d, const std::vector<float>& v) {
      return cudaMemcpyAsync(d, v.data(), sizeof(float) * ny, cudaMemcpyHostToDevice, c->stream);
    };
    auto upd = [&](double* d, const std::vector<double>& v) {
      return cudaMemcpyAsync(d, v.data(), sizeof(double) * ny, cudaMemcpyHostToDevice, c->stream);
    };
    CK(upf(c->crefp_f, crefp)); CK(upf(c->crefm_f, crefm)); CK(upf(c->crfp_f, crfp)); CK(upf(c->crfm_f, crfm));
    CK(upf(c->rhoref_f, rhoref)); CK(upf(c->rhorf_f, rhorf)); CK(upf(c->dPref_f, dPref)); CK(upf(c->Fvref_f, Fvref));
    CK(upd(c->meanrhs_d, mrhs)); CK(upd(c->meanshift_d, mshift));
    CK(upd(c->Hrefp_d, c->href_p)); CK(upd(c->Hrefm_d, c->href_m));
    CK(launch_make_shadows(c->cp, c->cm, c->Phi, c->Hcp, c->Hcm, shadows(c), mixed_refs(c), c->Hrefp_d, c->Hrefm_d, P,
                           c->nc, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->refs_valid = true;
    c->refs_dt = NAN;
    drop_graph(c);
  }
  if (!(c->refs_dt == dt)) {
    // the reference increments below need this dt's elimination factors
    if (!(c->cn_dt == dt) || c->cn_h.size() != 9 * kCnKinds * (size_t)ny) {
      int r = upload_cn(c, dt);
      if (r) return r;
    }
    // Rref(l, j) = dt alp_l (H_ref + D L_y c_ref): the reference part of the ion
    // CN right-hand side; stored solved, dC_ref = (I - s_l L_y)^-1 Rref, with the
    // substage's FP64 elimination factors (same as every ion line uses)
    std::vector<double> Rp(3 * (size_t)ny, 0.0), Rm(3 * (size_t)ny, 0.0);
    for (int l = 0; l < 3; ++l) {
      const double alp = kGam[l] + kZet[l];
      const double* A = c->cn_h.data() + ((size_t)(l * kCnKinds + 2) * 3 + 0) * ny;
      const double* Cp = c->cn_h.data() + ((size_t)(l * kCnKinds + 2) * 3 + 1) * ny;
      const double* M = c->cn_h.data() + ((size_t)(l * kCnKinds + 2) * 3 + 2) * ny;
      for (int ion = 0; ion < 2; ++ion) {
        const std::vector<double>& hr = ion == 0 ? c->href_p : c->href_m;
        const std::vector<double>& ly = ion == 0 ? c->lyc_p : c->lyc_m;
        double* out = (ion == 0 ? Rp.data() : Rm.data()) + (size_t)l * nyc;
        double d = 0.0;
        for (int j = 0; j < nyc; ++j) {
          const double r = dt * alp * (hr[j] + c->ph.D * ly[j]);
          d = (r - A[j] * d) * M[j];
          out[j] = d;
        }
        double x = 0.0;
        for (int j = nyc - 1; j >= 0; --j) {
          x = out[j] - Cp[j] * x;
          out[j] = x;
        }
      }
    }
    CK(cudaMemcpyAsync(c->Rrefp_d, Rp.data(), sizeof(double) * 3 * nyc, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->Rrefm_d, Rm.data(), sizeof(double) * 3 * nyc, cudaMemcpyHostToDevice, c->stream));
    std::vector<float2> Pp(3 * (size_t)nyc), Pm(3 * (size_t)nyc);
    for (size_t q = 0; q < Pp.size(); ++q) {
      const dfl a = df_split_host(Rp[q]), b = df_split_host(Rm[q]);
      Pp[q] = make_float2(a.h, a.l);
      Pm[q] = make_float2(b.h, b.l);
    }
    CK(cudaMemcpyAsync(c->dCp_f2, Pp.data(), sizeof(float2) * 3 * nyc, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->dCm_f2, Pm.data(), sizeof(float2) * 3 * nyc, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->refs_dt = dt;
  }
  return PNP_OK;
}

bool is_vel_field(int field) {
  return field == PNP_U || field == PNP_V || field == PNP_W || field == PNP_P || field == PNP_HU ||
         field == PNP_HV || field == PNP_HW;
}

void* field_ptr(pnp_ctx* c, int field) {
  switch (field) {
    case PNP_U: return c->u;
    case PNP_V: return c->v;
    case PNP_W: return c->w;
    case PNP_P: return c->p;
    case PNP_CP: return c->cp;
    case PNP_CM: return c->cm;
    case PNP_PHI: return c->Phi;
    case PNP_HU: return c->Hu;
    case PNP_HV: return c->Hv;
    case PNP_HW: return c->Hw;
    case PNP_HCP: return c->Hcp;
    case PNP_HCM: return c->Hcm;
    default: return nullptr;
  }
}

size_t field_count(const pnp_ctx* c, int field) {
  return (field == PNP_V || field == PNP_HV) ? c->nv : c->nc;
}

void drop_graph(pnp_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->graph_dt = NAN;
}

}  // namespace

extern "C" {

int pnp_workspace_bytes(int nx, int ny, int nz, int precision, size_t* out) {
  if (!out || (precision != PNP_FP64 && precision != PNP_MIXED)) return PNP_ERR_ARG;
  int r = check_grid(nx, ny, nz);
  if (r) return r;
  *out = carve(nullptr, nullptr, nx, ny, nz, precision);
  return PNP_OK;
}

int pnp_init_grid(pnp_ctx** out, int nx, int ny, int nz, double Lx, double Lz, double stretch, int precision,
                  void* ws, size_t bytes, void* stream) {
  if (!out || !ws || (precision != PNP_FP64 && precision != PNP_MIXED)) return PNP_ERR_ARG;
  if (!(Lx > 0) || !(Lz > 0) || !std::isfinite(stretch) || stretch < 0) return PNP_ERR_ARG;
  int r = check_grid(nx, ny, nz);
  if (r) return r;
  if (((uintptr_t)ws % kAlign) != 0) return PNP_ERR_WORKSPACE;
  if (bytes < carve(nullptr, nullptr, nx, ny, nz, precision)) return PNP_ERR_WORKSPACE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PNP_ERR_CUDA;
  pnp_ctx* c = new (std::nothrow) pnp_ctx();
  if (!c) return PNP_ERR_ARG;
  c->precision = precision;
  c->stream = (cudaStream_t)stream;
  c->ws = (char*)ws;
  c->ws_bytes = bytes;
  c->g.nx = nx;
  c->g.nz = nz;
  c->g.ny = ny;
  c->g.nyc = ny - 1;
  c->g.dx = Lx / nx;
  c->g.dz = Lz / nz;
  c->g.idx = 1.0 / c->g.dx;
  c->g.idz = 1.0 / c->g.dz;
  carve(c, c->ws, nx, ny, nz, precision);
  if (cudaMemsetAsync(c->ws, 0, bytes, c->stream) != cudaSuccess) { delete c; return PNP_ERR_CUDA; }
  // the TMA stencil needs whole x-rows of at most 512 floats in 128-byte multiples;
  // otherwise (or without the driver's tensor-map encoder) the cp.async tiles run
  if (precision == PNP_MIXED && rhs_tma_eligible(c->g))
    c->rhs_maps_ok = build_rhs_maps(&c->rhs_maps, fields<float>(c), shadows(c), c->g) == cudaSuccess;
  c->yf.assign(ny, 0.0);
  for (int j = 0; j < ny; ++j) {
    const double s = j * 2.0 / (ny - 1) - 1.0;
    c->yf[j] = stretch == 0.0 ? s : std::tanh(stretch * s) / std::tanh(stretch);
  }
  if (cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    pnp_destroy(c);
    return PNP_ERR_CUDA;
  }
  r = upload_metrics(c);
  if (r) { pnp_destroy(c); return r; }
  *out = c;
  return PNP_OK;
}

int pnp_set_yfaces(pnp_ctx* c, const double* yf, int ny) {
  if (!c || !yf || ny != c->g.ny) return PNP_ERR_ARG;
  for (int j = 0; j < ny; ++j) c->yf[j] = yf[j];
  c->have_state = false;
  return upload_metrics(c);
}

int pnp_set_params(pnp_ctx* c, double Re, double lam, double Sc, double V, double beta) {
  if (!c) return PNP_ERR_ARG;
  if (!(Re > 0) || !(lam > 0) || !(Sc > 0) || !std::isfinite(V) || !(beta >= 0) || !std::isfinite(Re) ||
      !std::isfinite(beta))
    return PNP_ERR_ARG;
  c->Re = Re; c->lam = lam; c->Sc = Sc; c->beta = beta;
  const double Uw = c->have_params ? c->ph.Uw : 1.0;
  c->ph.nu = 1.0 / Re;
  c->ph.D = 1.0 / (Re * Sc);
  c->ph.K = beta / (2.0 * Re * Re * Sc * lam * lam);
  c->ph.q = 1.0 / (2.0 * lam * lam);
  c->ph.V = V;
  c->ph.Uw = Uw;
  c->V_set = V;
  c->wall_map = false;   // uniform walls -V, +V
  c->edl_map = false;
  c->wall_off = 0.0;
  c->have_params = true;
  c->cn_dt = NAN;
  drop_graph(c);
  if (c->have_state) {   // parameters changed mid-run: the potential of the present ions under them
    int r = materialize(c);
    if (r) return r;
    CK(c->precision == PNP_FP64 ? potential_solve<double>(c) : potential_solve<float>(c));
    CK(cudaStreamSynchronize(c->stream));
    c->refs_valid = false;
  }
  return PNP_OK;
}

int pnp_set_wall_velocity(pnp_ctx* c, double Uw) {
  if (!c || !std::isfinite(Uw)) return PNP_ERR_ARG;
  if (!c->have_params) return PNP_ERR_STATE;
  c->ph.Uw = Uw;
  drop_graph(c);
  return PNP_OK;
}

int pnp_init_state(pnp_ctx* c, int ic_kind, uint64_t seed, double amp) {
  if (!c || (ic_kind != PNP_IC_LAMINAR && ic_kind != PNP_IC_PB) || !std::isfinite(amp)) return PNP_ERR_ARG;
  if (!c->have_params) return PNP_ERR_STATE;
  // bulk concentration of two Gouy-Chapman layers formed from c = 1:
  // c_b + 2 lam sqrt(c_b) (cosh(V/2) - 1) = 1
  const double bq = 2.0 * c->lam * (std::cosh(0.5 * c->ph.V) - 1.0);
  const double sq = 0.5 * (-bq + std::sqrt(bq * bq + 4.0));
  const double cb = sq * sq;
  const double kappa = std::sqrt(cb) / c->lam;
  cudaError_t e;
  if (c->precision == PNP_FP64)
    e = launch_init_fields<double>(fields<double>(c), c->g, metrics(c), c->ph, ic_kind, cb, kappa, seed, amp, c->yf_d, c->stream);
  else
    e = launch_init_fields<float>(fields<float>(c), c->g, metrics(c), c->ph, ic_kind, cb, kappa, seed, amp, c->yf_d, c->stream);
  if (e != cudaSuccess) return PNP_ERR_CUDA;
  if (amp != 0.0) {
    e = c->precision == PNP_FP64 ? pressure_projection<double>(c, 1.0, false) : pressure_projection<float>(c, 1.0, false);
    if (e != cudaSuccess) return PNP_ERR_CUDA;
  }
  e = c->precision == PNP_FP64 ? potential_solve<double>(c) : potential_solve<float>(c);
  if (e != cudaSuccess) return PNP_ERR_CUDA;
  c->have_state = true;
  c->fp64_fresh = true;
  c->refs_valid = false;
  c->time = 0.0;
  c->nstep = 0;
  return PNP_OK;
}

int pnp_field_size(pnp_ctx* c, int field, size_t* n) {
  if (!c || !n || field < 0 || field >= PNP_NFIELDS) return PNP_ERR_ARG;
  *n = field_count(c, field);
  return PNP_OK;
}

int pnp_set_state(pnp_ctx* c, int field, const void* src, int on_device) {
  if (!c || !src || field < 0 || field >= PNP_NFIELDS) return PNP_ERR_ARG;
  const size_t n = field_count(c, field);
  void* dst = field_ptr(c, field);
  const bool narrow = c->precision == PNP_MIXED && is_vel_field(field);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (c->precision == PNP_MIXED && !is_vel_field(field)) {
    int r = materialize(c);
    if (r) return r;
    c->refs_valid = false;
  }
  if (!narrow) {
    CK(cudaMemcpyAsync(dst, src, n * sizeof(double), kind, c->stream));
  } else {
    const double* s = (const double*)src;
    if (!on_device) {
      CK(cudaMemcpyAsync(c->stage, src, n * sizeof(double), kind, c->stream));
      s = c->stage;
    }
    CK(launch_convert<double, float>(s, (float*)dst, n, c->stream));
  }
  if (field <= PNP_PHI) c->have_state = true;
  return PNP_OK;
}

int pnp_get_state(pnp_ctx* c, int field, void* dst, int on_device) {
  if (!c || !dst || field < 0 || field >= PNP_NFIELDS) return PNP_ERR_ARG;
  const size_t n = field_count(c, field);
  const void* src = field_ptr(c, field);
  const bool narrow = c->precision == PNP_MIXED && is_vel_field(field);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  {
    int r = materialize(c);
    if (r) return r;
  }
  if (narrow) {
    double* tgt = on_device ? (double*)dst : c->stage;
    CK(launch_convert<float, double>((const float*)src, tgt, n, c->stream));
    if (!on_device) CK(cudaMemcpyAsync(dst, c->stage, n * sizeof(double), kind, c->stream));
  } else {
    CK(cudaMemcpyAsync(dst, src, n * sizeof(double), kind, c->stream));
  }
  if (!on_device) CK(cudaStreamSynchronize(c->stream));
  return PNP_OK;
}

int pnp_step(pnp_ctx* c, int nsteps, double dt) {
  if (!c || nsteps < 0 || !(dt > 0) || !std::isfinite(dt)) return PNP_ERR_ARG;
  if (!c->have_params || !c->have_state) return PNP_ERR_STATE;
  if (nsteps == 0) return PNP_OK;
  {
    int r = refresh_refs(c, dt);
    if (!r) r = prepare_tables(c, dt);
    if (r) return r;
  }
  if (c->precision == PNP_MIXED) c->fp64_fresh = false;
  if (c->stream == nullptr) {
    for (int n = 0; n < nsteps; ++n) CK(one_step(c, dt));
  } else {
    if (!c->gexec || c->graph_dt != dt) {
      drop_graph(c);
      cudaGraph_t graph = nullptr;
      CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
      cudaError_t e = one_step(c, dt);
      cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return PNP_ERR_CUDA;
      }
      e = cudaGraphInstantiate(&c->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) { c->gexec = nullptr; return PNP_ERR_CUDA; }
      c->graph_dt = dt;
    }
    for (int n = 0; n < nsteps; ++n) CK(cudaGraphLaunch(c->gexec, c->stream));
  }
  c->time += nsteps * dt;
  c->nstep += nsteps;
  c->last_dt = dt;
  return PNP_OK;
}

int pnp_step_adaptive(pnp_ctx* c, int nsteps, double dt_max, double cfl, int check_every, double* dts_out) {
  if (!c || nsteps < 0 || !(dt_max > 0) || !std::isfinite(dt_max) || !(cfl > 0) || cfl > 1 || check_every < 1)
    return PNP_ERR_ARG;
  if (!c->have_params || !c->have_state) return PNP_ERR_STATE;
  int rung = -1;   // ladder index of the current dt
  for (int done = 0; done < nsteps;) {
    pnp_diag d;
    const int st = pnp_diagnostics(c, &d);
    if (st != PNP_OK && st != PNP_ERR_CFL && st != PNP_ERR_DPHI) return st;
    const double lim = std::min(std::min(cfl * d.dt_cfl, cfl * d.dt_migration), 4.0 * cfl * d.dt_dielectric);
    int k = 0;
    if (lim < dt_max) k = (int)std::ceil(8.0 * std::log2(dt_max / lim) - 1e-12);
    if (rung >= 0 && k < rung - 1) k = rung - 1;   // grow by one rung at most
    if (k > 4096) return PNP_ERR_CFL;              // no usable dt (limits collapsed)
    rung = k;
    const double dt = dt_max * std::exp2(-k / 8.0);
    const int n = std::min(check_every, nsteps - done);
    const int r = pnp_step(c, n, dt);
    if (r) return r;
    if (dts_out)
      for (int q = 0; q < n; ++q) dts_out[done + q] = dt;
    done += n;
  }
  return PNP_OK;
}

int pnp_stats_reset(pnp_ctx* c) {
  if (!c) return PNP_ERR_ARG;
  CK(cudaMemsetAsync(c->stats_acc, 0, 12 * sizeof(double) * c->g.ny, c->stream));
  c->stats_n = 0;
  return PNP_OK;
}

int pnp_stats_sample(pnp_ctx* c) {
  if (!c) return PNP_ERR_ARG;
  if (!c->have_params || !c->have_state) return PNP_ERR_STATE;
  const bool shadows_now = c->precision == PNP_MIXED && c->refs_valid && !c->fp64_fresh;
  if (!shadows_now) {
    int r = materialize(c);
    if (r) return r;
  }
  StatSrc src{};
  src.u = c->u; src.v = c->v; src.w = c->w;
  src.vel_f32 = c->precision == PNP_MIXED;
  src.mixed = shadows_now;
  src.cp = c->cp; src.cm = c->cm; src.Phi = c->Phi;
  src.cpS = c->cpS; src.cpL = c->cpL; src.cmS = c->cmS; src.cmL = c->cmL; src.phiS = c->phiS;
  src.cref_p = c->cref64p_d; src.cref_m = c->cref64m_d; src.phi_ref = c->Phiref64_d;
  CK(launch_stats_sample(src, c->g, c->stats_acc, c->stream));
  ++c->stats_n;
  return PNP_OK;
}

int pnp_stats_get(pnp_ctx* c, double* mean_out, double* rms_out, double* cf_mean, long long* nsamples) {
  if (!c || !mean_out || !rms_out) return PNP_ERR_ARG;
  const int ny = c->g.ny, nyc = c->g.nyc;
  std::vector<double> a(12 * (size_t)ny);
  CK(cudaMemcpyAsync(a.data(), c->stats_acc, sizeof(double) * a.size(), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const double n = c->stats_n > 0 ? (double)c->stats_n : 1.0;
  for (int q = 0; q < 6; ++q) {
    const int planes = q == 1 ? ny : nyc;   // v on the faces
    for (int j = 0; j < ny; ++j) {
      double m = 0.0, r = 0.0;
      if (j < planes && c->stats_n > 0) {
        m = a[(size_t)(2 * q) * ny + j] / n;
        const double m2 = a[(size_t)(2 * q + 1) * ny + j] / n;
        r = std::sqrt(std::max(m2 - m * m, 0.0));
      }
      mean_out[(size_t)q * ny + j] = m;
      rms_out[(size_t)q * ny + j] = r;
    }
  }
  if (cf_mean) {
    const double Uw = c->ph.Uw;
    const double tb = c->ph.nu * (mean_out[0] + Uw) / c->h[0];
    const double tt = c->ph.nu * (Uw - mean_out[nyc - 1]) / c->h[nyc];
    *cf_mean = (c->stats_n > 0 && Uw != 0.0) ? (tb + tt) / (Uw * Uw) : 0.0;
  }
  if (nsamples) *nsamples = c->stats_n;
  return PNP_OK;
}

int pnp_set_wall_potential(pnp_ctx* c, const double* bottom, const double* top) {
  if (!c) return PNP_ERR_ARG;
  if (!c->have_params) return PNP_ERR_STATE;
  if ((bottom == nullptr) != (top == nullptr)) return PNP_ERR_ARG;
  c->edl_map = false;   // a map (or the uniform walls) replaces the wall model's offsets
  const size_t P = (size_t)c->g.nz * c->g.nx;
  if (!bottom) {
    c->wall_map = false;
    c->wall_off = 0.0;
    c->ph.V = c->V_set;
  } else {
    double sb = 0.0, st = 0.0;
    for (size_t q = 0; q < P; ++q) {
      if (!std::isfinite(bottom[q]) || !std::isfinite(top[q])) return PNP_ERR_ARG;
      sb += bottom[q];
      st += top[q];
    }
    const double Bm = sb / (double)P, Tm = st / (double)P;
    CK(cudaMemcpyAsync(c->wallB_d, bottom, sizeof(double) * P, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->wallT_d, top, sizeof(double) * P, cudaMemcpyHostToDevice, c->stream));
    // lift = Phi_0' + psi: the charge-free potential of the zero-mean wall
    // variations, one FP64 Dirichlet solve (the scratch of the pressure pipeline)
    const Metrics m = metrics(c);
    cplx<double>* spec = (cplx<double>*)c->spec;
    const cplx<double>* twx = (const cplx<double>*)c->twx_d;
    const cplx<double>* twp = (const cplx<double>*)c->twp_d;
    const cplx<double>* twz = (const cplx<double>*)c->twz_d;
    CK(launch_wall_lift_source(c->sreal, c->wallB_d, c->wallT_d, Bm, Tm, c->yc_d, c->g, c->stream));
    CK(launch_fft_x_fwd<double, double>(PoissonSrc::Plain, nullptr, nullptr, nullptr, nullptr, nullptr, c->sreal, 1.0,
                                        c->g, m, spec, twx, twp, c->stream));
    CK(spectral_solve<double>(c, spec, twz, false));
    CK(launch_fft_x_inv<double, double>(PoissonDst::Plain, spec, c->g, m, twx, twp, 0.0, c->lift64, c->stream));
    const double off = 0.5 * (Tm + Bm);
    CK(launch_wall_lift_finish(c->lift64, c->lift32, c->wallB_d, c->wallT_d, Bm, Tm, off, c->yc_d, c->g, c->stream));
    c->wall_map = true;
    c->wall_off = off;
    c->ph.V = 0.5 * (Tm - Bm);
  }
  drop_graph(c);
  if (c->have_state) {   // the potential of the current ions under the new walls
    int r = materialize(c);
    if (r) return r;
    const cudaError_t e = c->precision == PNP_FP64 ? potential_solve<double>(c) : potential_solve<float>(c);
    if (e != cudaSuccess) return PNP_ERR_CUDA;
    c->refs_valid = false;
  }
  CK(cudaStreamSynchronize(c->stream));
  return PNP_OK;
}

int pnp_set_scheme(pnp_ctx* c, int scheme) {
  if (!c || (scheme != PNP_SCHEME_CN && scheme != PNP_SCHEME_AF)) return PNP_ERR_ARG;
  if (c->scheme != scheme) drop_graph(c);
  c->scheme = scheme;
  c->af_dt = NAN;
  return PNP_OK;
}

int pnp_set_fusion(pnp_ctx* c, int on) {
  if (!c) return PNP_ERR_ARG;
  if ((on != 0) != c->fuse_cn) drop_graph(c);
  c->fuse_cn = on != 0;
  return PNP_OK;
}

int pnp_set_policy(pnp_ctx* c, int policy) {
  if (!c || (policy != PNP_POLICY_DEFAULT && policy != PNP_POLICY_FP64_SOLVES)) return PNP_ERR_ARG;
  if (policy != PNP_POLICY_DEFAULT && c->precision != PNP_MIXED) return PNP_ERR_UNSUPPORTED;
  if (c->policy != policy) drop_graph(c);
  c->policy = policy;
  return PNP_OK;
}

int pnp_set_limits(pnp_ctx* c, double cfl_max, double dphi_max) {
  if (!c || !(cfl_max > 0) || !(dphi_max > 0) || !std::isfinite(cfl_max) || !std::isfinite(dphi_max))
    return PNP_ERR_ARG;
  c->cfl_max = cfl_max;
  c->dphi_max = dphi_max;
  return PNP_OK;
}

namespace {
// Raw diagnostics record: device sums and status (written by the copies of a
// post), then the host-side values of the moment of the post.
struct DiagRaw {
  double h[kDiagOutSlots];
  int st[2];
  double wall_mean[2];   // plane-mean wall velocities (slip walls)
  double refN_p, refN_m, refH_p, refH_m;
  double time, last_dt;
  long long nstep;
  int from_shadows, slip_on;
};
static_assert(sizeof(DiagRaw) <= PNP_DIAG_RAW_BYTES, "raw diagnostics record");
}  // namespace

int pnp_diagnostics_post(pnp_ctx* c, void* raw_host) {
  if (!c || !raw_host) return PNP_ERR_ARG;
  if (!c->have_params || !c->have_state) return PNP_ERR_STATE;
  DiagRaw* R = static_cast<DiagRaw*>(raw_host);
  // mixed precision with valid shadows: straight from the FP32 fields and the
  // df ion state; otherwise from the FP64 arrays (current after pnp_init_state /
  // pnp_set_state, or brought up to date here)
  const bool from_shadows = c->precision == PNP_MIXED && c->refs_valid;
  if (!from_shadows) {
    int r = materialize(c);
    if (r) return r;
  }
  const DiagLimits lim{c->last_dt, c->cfl_max, c->dphi_max};
  cudaError_t e =
      from_shadows ? launch_diagnostics_mixed(fields<float>(c), shadows(c), c->crefp_f, c->crefm_f, c->dPref_f,
                                              c->diag_w, c->g, c->diag_partial, kDiagBlocks, c->diag_out,
                                              c->status_d, lim, c->stream)
      : c->precision == PNP_FP64
          ? launch_diagnostics<double>(fields<double>(c), c->g, metrics(c), c->ph, c->diag_partial, kDiagBlocks,
                                       c->diag_out, c->status_d, lim, c->stream)
          : launch_diagnostics<float>(fields<float>(c), c->g, metrics(c), c->ph, c->diag_partial, kDiagBlocks,
                                      c->diag_out, c->status_d, lim, c->stream);
  if (e != cudaSuccess) return PNP_ERR_CUDA;
  CK(cudaMemcpyAsync(R->h, c->diag_out, sizeof(R->h), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(R->st, c->status_d, sizeof(R->st), cudaMemcpyDeviceToHost, c->stream));
  if (c->slip_on) {
    const int P = c->g.nx * c->g.nz;
    cudaError_t e2 = c->precision == PNP_FP64
                         ? launch_mean_profile<double>((const double*)c->wall_u, 2, P, c->diag_out + kDiagOutSlots,
                                                       c->stream)
                         : launch_mean_profile<float>((const float*)c->wall_u, 2, P, c->diag_out + kDiagOutSlots,
                                                      c->stream);
    if (e2 != cudaSuccess) return PNP_ERR_CUDA;
    CK(cudaMemcpyAsync(R->wall_mean, c->diag_out + kDiagOutSlots, sizeof(R->wall_mean), cudaMemcpyDeviceToHost,
                       c->stream));
  }
  R->refN_p = c->refN_p;
  R->refN_m = c->refN_m;
  R->refH_p = c->refH_p;
  R->refH_m = c->refH_m;
  R->time = c->time;
  R->last_dt = c->last_dt;
  R->nstep = c->nstep;
  R->from_shadows = from_shadows ? 1 : 0;
  R->slip_on = c->slip_on ? 1 : 0;
  return PNP_OK;
}

int pnp_diagnostics_read(const pnp_ctx* c, const void* raw_host, pnp_diag* out) {
  if (!c || !raw_host || !out) return PNP_ERR_ARG;
  const DiagRaw* R = static_cast<const DiagRaw*>(raw_host);
  double h[kDiagOutSlots];
  std::memcpy(h, R->h, sizeof(h));
  if (R->from_shadows) {   // the reference parts of the ion numbers and of the explicit ion terms
    h[2] += R->refN_p;
    h[3] += R->refN_m;
    h[10] += R->refH_p;
    h[11] += R->refH_m;
  }
  const int st = R->st[1] ? R->st[1] : R->st[0];
  const double P = (double)c->g.nx * c->g.nz;
  const double ub = h[0] / P, ut = h[1] / P;
  const double Uw = c->ph.Uw;
  const double wb = R->slip_on ? R->wall_mean[0] : -Uw, wt = R->slip_on ? R->wall_mean[1] : Uw;
  std::memset(out, 0, sizeof(*out));
  out->tau_bot = c->ph.nu * (ub - wb) / c->h[0];
  out->tau_top = c->ph.nu * (wt - ut) / c->h[c->g.nyc];
  const double tau = 0.5 * (out->tau_bot + out->tau_top);
  out->cf = Uw != 0.0 ? 2.0 * tau / (Uw * Uw) : 0.0;
  out->re_tau = c->Re * std::sqrt(tau > 0 ? tau : 0.0);
  out->n_plus = h[2] * c->g.dx * c->g.dz;
  out->n_minus = h[3] * c->g.dx * c->g.dz;
  out->net_charge = out->n_plus - out->n_minus;
  // net ion flux out through the walls: the cell sums of -H_c telescope to the
  // wall-face fluxes (zero in the scheme, Fig. 1 caption)
  out->flux_plus = -h[10] * c->g.dx * c->g.dz;
  out->flux_minus = -h[11] * c->g.dx * c->g.dz;
  out->wall_flux = std::fabs(out->flux_plus) + std::fabs(out->flux_minus);
  out->cfl = R->last_dt * h[8];
  out->max_dphi = h[9];
  out->dt_cfl = h[8] > 0 ? 1.0 / h[8] : INFINITY;
  out->dt_migration = h[12] > 0 ? 1.0 / (c->ph.D * h[12]) : INFINITY;
  out->dt_dielectric = h[13] > 0 ? 1.0 / (c->ph.D * c->ph.q * h[13]) : INFINITY;
  out->max_div = h[4];
  out->ke = 0.5 * h[5] * c->g.dx * c->g.dz;
  out->time = R->time;
  out->nstep = R->nstep;
  out->status = st;
  out->precision = c->precision;
  return st;
}

int pnp_diagnostics(pnp_ctx* c, pnp_diag* out) {
  if (!c || !out) return PNP_ERR_ARG;
  DiagRaw raw{};
  int r = pnp_diagnostics_post(c, &raw);
  if (r) return r;
  CK(cudaStreamSynchronize(c->stream));
  return pnp_diagnostics_read(c, &raw, out);
}

int pnp_mean_profile(pnp_ctx* c, int field, double* out) {
  if (!c || !out || field < 0 || field >= PNP_NFIELDS) return PNP_ERR_ARG;
  const int planes = (field == PNP_V || field == PNP_HV) ? c->g.ny : c->g.nyc;
  const int P = c->g.nz * c->g.nx;
  {
    int r = materialize(c);
    if (r) return r;
  }
  const void* q = field_ptr(c, field);
  cudaError_t e = (c->precision == PNP_MIXED && is_vel_field(field))
                      ? launch_mean_profile<float>((const float*)q, planes, P, c->stage, c->stream)
                      : launch_mean_profile<double>((const double*)q, planes, P, c->stage, c->stream);
  if (e != cudaSuccess) return PNP_ERR_CUDA;
  CK(cudaMemcpyAsync(out, c->stage, sizeof(double) * planes, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PNP_OK;
}

int pnp_poisson(pnp_ctx* c, int bc, const double* rhs, double* x) {
  if (!c || !rhs || !x || (bc != PNP_NEUMANN && bc != PNP_DIRICHLET)) return PNP_ERR_ARG;
  const Metrics m = metrics(c);
  cplx<double>* spec = (cplx<double>*)c->spec;
  const cplx<double>* twx = (const cplx<double>*)c->twx_d;
  const cplx<double>* twp = (const cplx<double>*)c->twp_d;
  const cplx<double>* twz = (const cplx<double>*)c->twz_d;
  CK(launch_fft_x_fwd<double, double>(PoissonSrc::Plain, nullptr, nullptr, nullptr, nullptr, nullptr, rhs, 1.0, c->g,
                                      m, spec, twx, twp, c->stream));
  CK(spectral_solve<double>(c, spec, twz, bc == PNP_NEUMANN));
  CK(launch_fft_x_inv<double, double>(PoissonDst::Plain, spec, c->g, m, twx, twp, 0.0, x, c->stream));
  return PNP_OK;
}

int pnp_eval_explicit(pnp_ctx* c) {
  if (!c) return PNP_ERR_ARG;
  if (!c->have_params || !c->have_state) return PNP_ERR_STATE;
  const Stage st{1.0, 1.0, 0.0, 0.0};
  cudaError_t e;
  if (c->precision == PNP_FP64) {
    e = launch_rhs<double>(fields<double>(c), c->g, metrics(c), c->ph, st, c->stream);
  } else {
    int r = refresh_refs(c, std::isfinite(c->refs_dt) ? c->refs_dt : 1.0);
    if (r) return r;
    e = launch_mixed_rhs(fields<float>(c), shadows(c), mixed_refs(c), c->g, metrics_f(c), coef_f(c, st), rhs_maps(c),
                         c->status_d + 1, c->stream);
    c->fp64_fresh = false;
  }
  return e == cudaSuccess ? PNP_OK : PNP_ERR_CUDA;
}

int pnp_clear_status(pnp_ctx* c) {
  if (!c) return PNP_ERR_ARG;
  CK(cudaMemsetAsync(c->status_d, 0, 2 * sizeof(int), c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PNP_OK;
}

int pnp_selftest_wait_timeout(pnp_ctx* c, double limit_s) {
  if (!c || !(limit_s > 0.0) || limit_s > 10.0) return PNP_ERR_ARG;
  CK(launch_wait_selftest(c->status_d + 1, limit_s, c->stream));
  return pnp_status(c);
}

int pnp_status(pnp_ctx* c) {
  if (!c) return PNP_ERR_ARG;
  int st[2] = {0, 0};
  CK(cudaMemcpyAsync(st, c->status_d, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return st[1] ? st[1] : st[0];   // a copy timeout is sticky and takes precedence
}

int pnp_fp64_peak(pnp_ctx* c, double* flops) {
  if (!c || !flops) return PNP_ERR_ARG;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int iters = 4096;
  CK(launch_fp64_probe(c->probe_d, 64, kProbeBlocks, c->stream));   // warm-up
  CK(cudaEventRecord(e0, c->stream));
  CK(launch_fp64_probe(c->probe_d, iters, kProbeBlocks, c->stream));
  CK(cudaEventRecord(e1, c->stream));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *flops = 2.0 * 8.0 * iters * (double)kProbeBlocks * 256.0 / (ms * 1e-3);
  return PNP_OK;
}

}  // extern "C"

namespace {

// Kernel launches of one step: capture the step into a graph (nothing runs)
// and count its kernel nodes.  -1 when the context has no stream to capture on.
int count_step_kernels(pnp_ctx* c, double dt) {
  if (c->stream == nullptr) return -1;
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) return -1;
  const cudaError_t e = one_step(c, dt);
  const cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return -1;
  }
  size_t n = 0;
  int kernels = -1;
  if (cudaGraphGetNodes(graph, nullptr, &n) == cudaSuccess) {
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(graph, nodes.data(), &n) == cudaSuccess) {
      kernels = 0;
      for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
      }
    }
  }
  cudaGraphDestroy(graph);
  return kernels;
}

}  // namespace

extern "C" {

int pnp_profile(pnp_ctx* c, int nsteps, double dt, double* ms_out, int nsites, int* launches_per_step) {
  if (!c || !ms_out || nsites < PNP_PROFILE_SITES || nsteps < 1 || !(dt > 0)) return PNP_ERR_ARG;
  if (!c->have_params || !c->have_state) return PNP_ERR_STATE;
  {
    int r = refresh_refs(c, dt);
    if (!r) r = prepare_tables(c, dt);
    if (r) return r;
  }
  if (c->precision == PNP_MIXED) c->fp64_fresh = false;
  const int kernels = count_step_kernels(c, dt);
  Prof prof;
  for (int i = 0; i < Prof::kMax; ++i) CK(cudaEventCreate(&prof.ev[i]));
  for (int i = 0; i < PNP_PROFILE_SITES; ++i) ms_out[i] = 0.0;
  c->prof = &prof;
  int rc = PNP_OK;
  for (int n = 0; n < nsteps && rc == PNP_OK; ++n) {
    for (int l = 0; l < 3 && rc == PNP_OK; ++l) {
      prof.n = 0;
      cudaError_t e = c->precision == PNP_FP64 ? substage<double>(c, dt, l) : substage_mixed(c, dt, l);
      if (e != cudaSuccess || prof.n != PNP_PROFILE_SITES + 1 || cudaStreamSynchronize(c->stream) != cudaSuccess) {
        rc = PNP_ERR_CUDA;
        break;
      }
      for (int i = 0; i < PNP_PROFILE_SITES; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, prof.ev[i], prof.ev[i + 1]) != cudaSuccess) rc = PNP_ERR_CUDA;
        ms_out[i] += ms;
      }
    }
  }
  c->prof = nullptr;
  for (int i = 0; i < Prof::kMax; ++i) cudaEventDestroy(prof.ev[i]);
  if (rc == PNP_OK) {
    c->time += nsteps * dt;
    c->nstep += nsteps;
  }
  if (launches_per_step) *launches_per_step = kernels;
  return rc;
}

int pnp_timeline(pnp_ctx* c, double dt, int in_graph, int cap, int* site_out, int* stream_out, double* t_ms_out,
                 int* n_out) {
  if (!c || !site_out || !stream_out || !t_ms_out || !n_out || cap < 1 || !(dt > 0)) return PNP_ERR_ARG;
  if (in_graph && !c->stream) return PNP_ERR_ARG;   // a capture needs a stream of its own
  if (!c->have_params || !c->have_state) return PNP_ERR_STATE;
  {
    int r = refresh_refs(c, dt);
    if (!r) r = prepare_tables(c, dt);
    if (r) return r;
  }
  if (c->precision == PNP_MIXED) c->fp64_fresh = false;
  CK(cudaStreamSynchronize(c->stream));
  Prof prof;
  prof.timeline = true;
  prof.external = in_graph != 0;
  for (int i = 0; i < Prof::kMax; ++i) CK(cudaEventCreate(&prof.ev[i]));
  c->prof = &prof;
  int rc = PNP_OK;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (in_graph && cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) rc = PNP_ERR_CUDA;
  for (int l = 0; l < 3 && rc == PNP_OK; ++l) {
    cudaError_t e = c->precision == PNP_FP64 ? substage<double>(c, dt, l) : substage_mixed(c, dt, l);
    if (e != cudaSuccess) rc = PNP_ERR_CUDA;
  }
  if (in_graph) {
    // the traced step as one graph (the events as its event-record nodes), launched once
    const cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
    if (rc == PNP_OK && (e2 != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess ||
                         cudaGraphLaunch(exec, c->stream) != cudaSuccess))
      rc = PNP_ERR_CUDA;
    cudaGetLastError();
  }
  c->prof = nullptr;
  if (rc == PNP_OK && (cudaStreamSynchronize(c->stream) != cudaSuccess || cudaStreamSynchronize(c->aux) != cudaSuccess))
    rc = PNP_ERR_CUDA;
  int n = 0;
  for (int i = 0; i < prof.n && n < cap && rc == PNP_OK; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, prof.ev[0], prof.ev[i]) != cudaSuccess) {
      rc = PNP_ERR_CUDA;
      break;
    }
    site_out[n] = prof.site[i];
    stream_out[n] = prof.on_aux[i];
    t_ms_out[n] = ms;
    ++n;
  }
  *n_out = n;
  for (int i = 0; i < Prof::kMax; ++i) cudaEventDestroy(prof.ev[i]);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (rc == PNP_OK) {
    c->time += dt;
    c->nstep += 1;
  }
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner: time candidate launch shapes of the stencil, CN-sweep, spectral
// y-solve and z-transform kernels on this context's grid (CUDA events, best of
// a few repetitions) and keep the fastest.  Runs on the workspace contents and
// overwrites them: call it before pnp_init_state / pnp_set_state.
// ---------------------------------------------------------------------------
namespace {

template <typename F>
float time_launches(pnp_ctx* c, F&& f, int reps) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  f();   // warm-up (and launch-shape validation)
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(a, c->stream);
    f();
    cudaEventRecord(b, c->stream);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (cudaGetLastError() != cudaSuccess) return 1e30f;
  return best;
}

}  // namespace

extern "C" {

int pnp_autotune(pnp_ctx* c, double dt, int* cfg_out, double* ms_out) {
  if (!c || !cfg_out || !(dt > 0)) return PNP_ERR_ARG;
  if (!c->have_params) return PNP_ERR_STATE;
  if (c->cn_dt != dt) {
    int r = upload_cn(c, dt);
    if (r) return r;
  }
  if (c->precision == PNP_MIXED) {
    c->fp64_fresh = true;
    c->refs_valid = false;
    int r = refresh_refs(c, dt);
    if (r) return r;
  }
  {
    int r = prepare_tables(c, dt);
    if (r) return r;
  }
  const Stage st{dt, kGam[0], kZet[0], kGam[0] + kZet[0]};
  const int reps = 3;
  float best[4] = {1e30f, 1e30f, 1e30f, 1e30f};
  int pick[4] = {32, 128, 64, 32};
  // 1: stencil block shape
  for (int bx : {32, 64, 128, 16}) {
    // FP64: block x-extents; mixed: 128 = TMA rows (when available), 64 / 32 / 16 = cp.async tiles
    if (c->precision == PNP_FP64 && bx > 2 * c->g.nx && bx != 32) continue;
    if (c->precision == PNP_MIXED && bx == 128 && !c->rhs_maps_ok) continue;
    c->g.lc_rhs_bx = bx;
    float t = time_launches(c, [&] {
      if (c->precision == PNP_FP64) launch_rhs<double>(fields<double>(c), c->g, metrics(c), c->ph, st, c->stream);
      else launch_mixed_rhs(fields<float>(c), shadows(c), mixed_refs(c), c->g, metrics_f(c), coef_f(c, st), rhs_maps(c),
                            c->status_d + 1, c->stream);
    }, reps);
    if (t < best[0]) { best[0] = t; pick[0] = bx; }
  }
  c->g.lc_rhs_bx = pick[0];
  // 2: CN sweep block size
  for (int T : {32, 64, 128, 256}) {   // mixed: 32 = shared-memory line tiles
    c->g.lc_cn = T;
    float t = time_launches(c, [&] {
      if (c->precision == PNP_FP64)
        launch_cn_solves<double>(fields<double>(c), c->g, cn_rows(c, 0, 0), cn_rows(c, 0, 1), cn_rows(c, 0, 2), c->stream);
      else
        launch_mixed_cn(fields<float>(c), shadows(c), mixed_refs(c), c->g, cn_rows_f(c, 0, 0), cn_rows_f(c, 0, 1),
                        cn_rows_f(c, 0, 2), 0, kCnIons | kCnVelocity, c->stream);
    }, reps);
    if (t < best[1]) { best[1] = t; pick[1] = T; }
  }
  c->g.lc_cn = pick[1];
  // 3: spectral y-solve block size, 4: z-transform threads per column
  const double scale = 1.0 / ((double)c->g.nx * (double)c->g.nz);
  for (int T : {16, 32, 64, 128}) {   // mixed: 16 = shared-memory tiles
    c->g.lc_spec = T;
    float t = time_launches(c, [&] {
      if (c->precision == PNP_FP64)
        launch_spec_thomas<double>((cplx<double>*)c->spec, c->dscr, c->spc_cprD, c->spc_invD, yrows(c, false), c->g,
                                   scale, false, c->stream);
      else
        launch_spec_thomas_df((cplx<float>*)c->spec, c->dscr, spec_df(c, false), c->spc_cprD, c->spc_invD,
                              yrows(c, false), c->g, scale, false, c->stream);
    }, reps);
    if (t < best[2]) { best[2] = t; pick[2] = T; }
  }
  c->g.lc_spec = pick[2];
  for (int ty : {8, 16, 32, 64}) {
    if (ty > 8 && ty > c->g.nz / 4) continue;
    c->g.lc_fftz_ty = ty;
    float t = time_launches(c, [&] {
      if (c->precision == PNP_FP64)
        launch_fft_z<double>((cplx<double>*)c->spec, (const cplx<double>*)c->twz_d, c->g, false, c->stream);
      else
        launch_fft_z<float>((cplx<float>*)c->spec, (const cplx<float>*)c->twz_f, c->g, false, c->stream);
    }, reps);
    if (t < best[3]) { best[3] = t; pick[3] = ty; }
  }
  c->g.lc_fftz_ty = pick[3];
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaGetLastError());
  // 5: the whole step.  Timed alone, the sites cannot show how their launch
  // shapes interact inside a step (the two streams share HBM and SMs), and
  // candidates a few percent apart alone can order differently there.  So each
  // choice is re-checked, one code at a time (coordinate descent from the
  // per-site picks), on the time of whole steps from a Poisson-Boltzmann
  // initial state (best of three runs of 16 steps), and a candidate replaces
  // the pick only if it is faster by more than 1% (closer calls are noise
  // between runs and boxes).
  {
    int r = pnp_init_state(c, PNP_IC_PB, 1, 1e-2);
    if (r) return r;
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    auto step_ms = [&]() -> float {
      drop_graph(c);
      if (pnp_step(c, 2, dt) != PNP_OK) return 1e30f;   // warm-up (and graph capture)
      constexpr int kSteps = 16;
      float bestm = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(a, c->stream);
        if (pnp_step(c, kSteps, dt) != PNP_OK) return 1e30f;
        cudaEventRecord(b, c->stream);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        bestm = std::min(bestm, ms / kSteps);
      }
      return bestm;
    };
    auto set = [&](int i, int v) {
      int* f[4] = {&c->g.lc_rhs_bx, &c->g.lc_cn, &c->g.lc_spec, &c->g.lc_fftz_ty};
      *f[i] = v;
    };
    float cur = step_ms();
    const std::vector<int> cands[4] = {{32, 64, 128, 16}, {32, 64, 128, 256}, {16, 32, 64, 128}, {8, 16, 32, 64}};
    for (int i = 0; i < 4; ++i) {
      for (int v : cands[i]) {
        if (v == pick[i]) continue;
        if (i == 0 && c->precision == PNP_FP64 && v > 2 * c->g.nx && v != 32) continue;
        if (i == 0 && c->precision == PNP_MIXED && v == 128 && !c->rhs_maps_ok) continue;
        if (i == 3 && v > 8 && v > c->g.nz / 4) continue;
        set(i, v);
        const float t = step_ms();
        if (t < 0.99f * cur) {
          cur = t;
          pick[i] = v;
        }
        set(i, pick[i]);
      }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    drop_graph(c);
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaGetLastError());
  }
  for (int i = 0; i < 4; ++i) {
    cfg_out[i] = pick[i];
    if (ms_out) ms_out[i] = best[i];
  }
  c->have_state = false;   // the timing launches overwrote the workspace
  drop_graph(c);
  return PNP_OK;
}

int pnp_set_launch_config(pnp_ctx* c, const int* cfg) {
  if (!c || !cfg) return PNP_ERR_ARG;
  const int bx = cfg[0], cn = cfg[1], sp = cfg[2], ty = cfg[3];
  if (!(bx == 16 || bx == 32 || bx == 64 || bx == 128)) return PNP_ERR_ARG;
  if (cn < 32 || cn > 1024 || (cn & (cn - 1))) return PNP_ERR_ARG;
  if (sp < 16 || sp > 1024 || (sp & (sp - 1))) return PNP_ERR_ARG;
  if (ty < 1 || ty > 64) return PNP_ERR_ARG;
  c->g.lc_rhs_bx = bx;
  c->g.lc_cn = cn;
  c->g.lc_spec = sp;
  c->g.lc_fftz_ty = ty;
  drop_graph(c);
  return PNP_OK;
}

int pnp_get_launch_config(pnp_ctx* c, int* cfg) {
  if (!c || !cfg) return PNP_ERR_ARG;
  cfg[0] = c->g.lc_rhs_bx ? c->g.lc_rhs_bx : (c->precision == PNP_MIXED && c->g.nx >= 64 ? 64 : 32);
  cfg[1] = c->g.lc_cn ? c->g.lc_cn : 128;
  cfg[2] = c->g.lc_spec ? c->g.lc_spec : 64;
  cfg[3] = c->g.lc_fftz_ty ? c->g.lc_fftz_ty : 32;
  return PNP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Ensemble of independent cases (uneven grids and parameters) advanced by ONE
// CUDA graph launch per step: the capture forks every case onto its own
// stream branch, so the cases' kernels overlap on the GPU.
// ---------------------------------------------------------------------------
struct pnp_ensemble {
  std::vector<pnp_ctx*> cases;
  std::vector<cudaStream_t> branch;   // private capture branch per case
  cudaStream_t stream = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t exec = nullptr;
  std::vector<double> dts;
};

extern "C" {

int pnp_ensemble_create(pnp_ensemble** out, pnp_ctx* const* cases, int ncases, void* stream) {
  if (!out || !cases || ncases < 1 || !stream) return PNP_ERR_ARG;
  for (int i = 0; i < ncases; ++i) {
    if (!cases[i]) return PNP_ERR_ARG;
    for (int k = 0; k < i; ++k)
      if (cases[k] == cases[i]) return PNP_ERR_ARG;
  }
  pnp_ensemble* e = new (std::nothrow) pnp_ensemble();
  if (!e) return PNP_ERR_ARG;
  e->cases.assign(cases, cases + ncases);
  e->stream = (cudaStream_t)stream;
  e->join.resize(ncases, nullptr);
  e->branch.resize(ncases, nullptr);
  bool ok = cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < ncases && ok; ++i) ok = cudaEventCreateWithFlags(&e->join[i], cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < ncases && ok; ++i) ok = cudaStreamCreateWithFlags(&e->branch[i], cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) {
    pnp_ensemble_destroy(e);
    return PNP_ERR_CUDA;
  }
  *out = e;
  return PNP_OK;
}

int pnp_ensemble_step(pnp_ensemble* e, int nsteps, const double* dt) {
  if (!e || !dt || nsteps < 0) return PNP_ERR_ARG;
  const int n = (int)e->cases.size();
  for (int i = 0; i < n; ++i) {
    pnp_ctx* c = e->cases[i];
    if (!(dt[i] > 0) || !std::isfinite(dt[i])) return PNP_ERR_ARG;
    if (!c->have_params || !c->have_state) return PNP_ERR_STATE;
  }
  if (nsteps == 0) return PNP_OK;
  bool recapture = !e->exec || (int)e->dts.size() != n;
  for (int i = 0; i < n; ++i) {
    pnp_ctx* c = e->cases[i];
    const bool had_refs = c->refs_valid;
    int r = refresh_refs(c, dt[i]);
    if (!r) r = prepare_tables(c, dt[i]);
    if (r) return r;
    if (c->precision == PNP_MIXED) c->fp64_fresh = false;
    if (!had_refs || (!recapture && e->dts[i] != dt[i])) recapture = true;
  }
  // finish every case's pending work (uploads, earlier steps) before the ensemble stream runs
  for (int i = 0; i < n; ++i) CK(cudaStreamSynchronize(e->cases[i]->stream));
  if (recapture) {
    if (e->exec) cudaGraphExecDestroy(e->exec);
    e->exec = nullptr;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeRelaxed));
    cudaError_t err = cudaEventRecord(e->fork, e->stream);
    for (int i = 0; i < n && err == cudaSuccess; ++i) {
      pnp_ctx* c = e->cases[i];
      cudaStream_t own = c->stream;
      c->stream = e->branch[i];   // the case's launches go to its capture branch
      err = cudaStreamWaitEvent(c->stream, e->fork, 0);
      if (err == cudaSuccess) err = one_step(c, dt[i]);
      if (err == cudaSuccess) err = cudaEventRecord(e->join[i], c->stream);
      if (err == cudaSuccess) err = cudaStreamWaitEvent(e->stream, e->join[i], 0);
      c->stream = own;
    }
    cudaError_t err2 = cudaStreamEndCapture(e->stream, &graph);
    if (err != cudaSuccess || err2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return PNP_ERR_CUDA;
    }
    err = cudaGraphInstantiate(&e->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (err != cudaSuccess) {
      e->exec = nullptr;
      return PNP_ERR_CUDA;
    }
    e->dts.assign(dt, dt + n);
  }
  for (int s = 0; s < nsteps; ++s) CK(cudaGraphLaunch(e->exec, e->stream));
  // later work issued on a case's own stream must follow the ensemble's steps
  CK(cudaEventRecord(e->fork, e->stream));
  for (int i = 0; i < n; ++i) {
    if (e->cases[i]->stream) CK(cudaStreamWaitEvent(e->cases[i]->stream, e->fork, 0));
    else CK(cudaStreamSynchronize(e->stream));
    e->cases[i]->time += nsteps * dt[i];
    e->cases[i]->nstep += nsteps;
    e->cases[i]->last_dt = dt[i];
  }
  return PNP_OK;
}

void pnp_ensemble_destroy(pnp_ensemble* e) {
  if (!e) return;
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->fork) cudaEventDestroy(e->fork);
  for (cudaEvent_t ev : e->join)
    if (ev) cudaEventDestroy(ev);
  for (cudaStream_t st : e->branch)
    if (st) cudaStreamDestroy(st);
  delete e;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Learned wall model: MLP workspace and the coupling to a coarse context.
// ---------------------------------------------------------------------------
constexpr int kMlpMaxPartial = 320;

struct pnp_mlp {
  MlpBufs b{};
  int max_batch = 0;
  int max_partial = 64;   // weight-gradient CTAs: two per SM (at most kMlpMaxPartial)
  size_t nparam = 0;
  cudaStream_t stream = nullptr;
  int t_adam = 0;
};

namespace {

size_t mlp_carve(pnp_mlp* m, char* base, int max_batch) {
  Bump bp{base};
  const MlpDims d = mlp_dims();
  const size_t np = d.nparam, B = (size_t)max_batch;
  MlpBufs b{};
  b.param = bp.take<float>(np);
  b.wimg = bp.take<__nv_bfloat16>(mlp_images().total);
  b.grad = bp.take<float>(np);
  b.m = bp.take<float>(np);
  b.v = bp.take<float>(np);
  b.act[0] = bp.take<float>(B * kMlpIn);
  for (int l = 0; l < kMlpLayers; ++l) b.act[l + 1] = bp.take<float>(B * d.out[l]);
  b.dact = bp.take<float>(B * kMlpHidden);
  b.dact2 = bp.take<float>(B * kMlpHidden);
  b.partial = bp.take<float>(kMlpMaxPartial * (size_t)(kMlpHidden * kMlpHidden + kMlpHidden));
  b.loss = bp.take<float>(128);
  b.in_shift = bp.take<float>(kMlpIn);
  b.in_scale = bp.take<float>(kMlpIn);
  b.out_shift = bp.take<float>(kMlpOut);
  b.out_scale = bp.take<float>(kMlpOut);
  b.err = bp.take<int>(4);
  if (m) {
    m->b = b;
    m->nparam = np;
  }
  return bp.off + kAlign;
}

uint64_t sm64_host(uint64_t seed, uint64_t n) {
  uint64_t x = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

WallMap wall_map(const pnp_ctx* f, const pnp_ctx* c, int* err) {
  WallMap wm{};
  *err = PNP_ERR_ARG;
  if (f->g.nx % c->g.nx || f->g.nz % c->g.nz || f->g.nyc % c->g.nyc) return wm;
  wm.nx_f = f->g.nx; wm.nz_f = f->g.nz; wm.nyc_f = f->g.nyc;
  wm.nx_c = c->g.nx; wm.nz_c = c->g.nz; wm.nyc_c = c->g.nyc;
  wm.rx = f->g.nx / c->g.nx; wm.rz = f->g.nz / c->g.nz; wm.ry = f->g.nyc / c->g.nyc;
  for (int jc = 0; jc <= c->g.nyc; ++jc)
    if (std::fabs(c->yf[jc] - f->yf[jc * wm.ry]) > 1e-12) return wm;   // coarse faces must be fine faces
  *err = PNP_OK;
  return wm;
}

}  // namespace

extern "C" {

int pnp_mlp_param_count(size_t* out) {
  if (!out) return PNP_ERR_ARG;
  *out = mlp_dims().nparam;
  return PNP_OK;
}

int pnp_mlp_workspace_bytes(int max_batch, size_t* out) {
  if (!out || max_batch < 1) return PNP_ERR_ARG;
  *out = mlp_carve(nullptr, nullptr, max_batch);
  return PNP_OK;
}

int pnp_mlp_create(pnp_mlp** out, int max_batch, void* ws, size_t bytes, void* stream, uint64_t seed) {
  if (!out || !ws || max_batch < 1) return PNP_ERR_ARG;
  if (((uintptr_t)ws % kAlign) != 0 || bytes < mlp_carve(nullptr, nullptr, max_batch)) return PNP_ERR_WORKSPACE;
  pnp_mlp* m = new (std::nothrow) pnp_mlp();
  if (!m) return PNP_ERR_ARG;
  m->max_batch = max_batch;
  m->stream = (cudaStream_t)stream;
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
      m->max_partial = std::min(2 * sms, kMlpMaxPartial);
  }
  mlp_carve(m, (char*)ws, max_batch);
  // weights U(-a, a), a = sqrt(6 / fan_in) from SplitMix64; biases 0; unit normalisation
  const MlpDims d = mlp_dims();
  std::vector<float> p(d.nparam, 0.f);
  for (int l = 0; l < kMlpLayers; ++l) {
    const double a = std::sqrt(6.0 / d.in[l]);
    for (size_t e = 0; e < (size_t)d.in[l] * d.out[l]; ++e) {
      const double u01 = (double)(sm64_host(seed, d.woff[l] + e) >> 11) * 0x1p-53;
      p[d.woff[l] + e] = (float)(a * (2.0 * u01 - 1.0));
    }
  }
  std::vector<float> ones(kMlpIn, 1.f), zeros(kMlpIn, 0.f);
  bool ok = cudaMemsetAsync(ws, 0, bytes, m->stream) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(m->b.param, p.data(), sizeof(float) * d.nparam, cudaMemcpyHostToDevice, m->stream) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(m->b.in_scale, ones.data(), sizeof(float) * kMlpIn, cudaMemcpyHostToDevice, m->stream) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(m->b.out_scale, ones.data(), sizeof(float) * kMlpOut, cudaMemcpyHostToDevice, m->stream) == cudaSuccess;
  ok = ok && mlp_sync_bf16(m->b, d.nparam, m->stream) == cudaSuccess;
  ok = ok && cudaStreamSynchronize(m->stream) == cudaSuccess;
  if (!ok) { delete m; return PNP_ERR_CUDA; }
  *out = m;
  return PNP_OK;
}

int pnp_mlp_get_params(pnp_mlp* m, float* host, size_t n) {
  if (!m || !host || n != m->nparam) return PNP_ERR_ARG;
  CK(cudaMemcpyAsync(host, m->b.param, sizeof(float) * n, cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return PNP_OK;
}

int pnp_mlp_set_params(pnp_mlp* m, const float* host, size_t n) {
  if (!m || !host || n != m->nparam) return PNP_ERR_ARG;
  CK(cudaMemcpyAsync(m->b.param, host, sizeof(float) * n, cudaMemcpyHostToDevice, m->stream));
  CK(cudaMemsetAsync(m->b.m, 0, sizeof(float) * n, m->stream));
  CK(cudaMemsetAsync(m->b.v, 0, sizeof(float) * n, m->stream));
  CK(mlp_sync_bf16(m->b, n, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  m->t_adam = 0;
  return PNP_OK;
}

int pnp_mlp_set_normalization(pnp_mlp* m, const float* in_shift, const float* in_scale, const float* out_shift,
                              const float* out_scale) {
  if (!m || !in_shift || !in_scale || !out_shift || !out_scale) return PNP_ERR_ARG;
  CK(cudaMemcpyAsync(m->b.in_shift, in_shift, sizeof(float) * kMlpIn, cudaMemcpyHostToDevice, m->stream));
  CK(cudaMemcpyAsync(m->b.in_scale, in_scale, sizeof(float) * kMlpIn, cudaMemcpyHostToDevice, m->stream));
  CK(cudaMemcpyAsync(m->b.out_shift, out_shift, sizeof(float) * kMlpOut, cudaMemcpyHostToDevice, m->stream));
  CK(cudaMemcpyAsync(m->b.out_scale, out_scale, sizeof(float) * kMlpOut, cudaMemcpyHostToDevice, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return PNP_OK;
}

int pnp_mlp_set_skip(pnp_mlp* m, int out_col, int in_col) {
  if (!m || out_col >= kMlpOut || in_col >= kMlpIn || (out_col >= 0 && in_col < 0)) return PNP_ERR_ARG;
  m->b.skip_out = out_col < 0 ? -1 : out_col;
  m->b.skip_in = out_col < 0 ? -1 : in_col;
  return PNP_OK;
}

int pnp_mlp_forward(pnp_mlp* m, const float* X, int B, float* Y) {
  if (!m || !X || !Y || B < 1 || B > m->max_batch) return PNP_ERR_ARG;
  CK(mlp_forward(m->b, X, B, Y, m->stream));
  return PNP_OK;
}

int pnp_mlp_gradient(pnp_mlp* m, const float* X, const float* T, int B, float* grad_host, float* loss_host) {
  if (!m || !X || !T || B < 1 || B > m->max_batch) return PNP_ERR_ARG;
  CK(mlp_forward(m->b, X, B, nullptr, m->stream));
  CK(mlp_backward(m->b, X, T, B, m->max_partial, m->stream));
  if (grad_host) CK(cudaMemcpyAsync(grad_host, m->b.grad, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost, m->stream));
  if (loss_host) CK(cudaMemcpyAsync(loss_host, m->b.loss + 120, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return PNP_OK;
}

int pnp_mlp_train_step(pnp_mlp* m, const float* X, const float* T, int B, float lr, float* loss_host) {
  if (!m || !X || !T || B < 1 || B > m->max_batch || !(lr > 0)) return PNP_ERR_ARG;
  CK(mlp_forward(m->b, X, B, nullptr, m->stream));
  CK(mlp_backward(m->b, X, T, B, m->max_partial, m->stream));
  m->t_adam += 1;
  CK(mlp_adam(m->b, m->nparam, lr, 0.9f, 0.999f, 1e-8f, m->t_adam, m->stream));
  if (loss_host) {
    CK(cudaMemcpyAsync(loss_host, m->b.loss + 120, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
  }
  return PNP_OK;
}

int pnp_mlp_status(pnp_mlp* m) {
  if (!m) return PNP_ERR_ARG;
  int st = 0;
  CK(cudaMemcpyAsync(&st, m->b.err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return st;
}

void pnp_mlp_destroy(pnp_mlp* m) { delete m; }

int pnp_wall_features(pnp_ctx* c, int ncells, float* X) {
  if (!c || !X || ncells < 1 || ncells > 8 || ncells > c->g.nyc) return PNP_ERR_ARG;
  if (!c->have_state) return PNP_ERR_STATE;
  IonView iv{};
  int r = ion_view(c, &iv);
  if (r) return r;
  const double* lift = c->edl_map ? c->lift64 : nullptr;   // features see the walls -V, +V alone
  cudaError_t e = c->precision == PNP_FP64
                      ? launch_wall_features<double>((const double*)c->u, (const double*)c->w, iv, c->yc_d, c->g,
                                                     c->ph.V, c->ph.Uw, ncells, lift, X, c->stream)
                      : launch_wall_features<float>((const float*)c->u, (const float*)c->w, iv, c->yc_d, c->g,
                                                    c->ph.V, c->ph.Uw, ncells, lift, X, c->stream);
  return e == cudaSuccess ? PNP_OK : PNP_ERR_CUDA;
}

int pnp_restrict_state(pnp_ctx* f, pnp_ctx* c) {
  if (!f || !c || f == c) return PNP_ERR_ARG;
  if (!f->have_state || !c->have_params) return PNP_ERR_STATE;
  int err = 0;
  const WallMap wm = wall_map(f, c, &err);
  if (err) return err;
  int r = materialize(f);
  if (r) return r;
  double* dyf = nullptr;
  // fine cell heights: reuse the fine context's staging area tail (ny values) as scratch
  dyf = f->stage + f->nv - f->g.ny;
  CK(cudaMemcpyAsync(dyf, f->dy.data(), sizeof(double) * f->g.nyc, cudaMemcpyHostToDevice, f->stream));
  const int fields_[7] = {PNP_U, PNP_V, PNP_W, PNP_P, PNP_CP, PNP_CM, PNP_PHI};
  for (int q = 0; q < 7; ++q) {
    const int fld = fields_[q];
    const void* src = field_ptr(f, fld);
    const bool vf = fld == PNP_V;
    double* out = f->sreal;   // fine scratch is large enough for any coarse field
    cudaError_t e;
    if (f->precision == PNP_MIXED && is_vel_field(fld)) e = launch_restrict<float>((const float*)src, dyf, wm, out, vf, f->stream);
    else e = launch_restrict<double>((const double*)src, dyf, wm, out, vf, f->stream);
    if (e != cudaSuccess) return PNP_ERR_CUDA;
    CK(cudaStreamSynchronize(f->stream));
    r = pnp_set_state(c, fld, out, 1);
    if (r) return r;
    CK(cudaStreamSynchronize(c->stream));
  }
  // the coarse run starts with no stored explicit terms
  for (int fld : {PNP_HU, PNP_HV, PNP_HW}) CK(cudaMemsetAsync(field_ptr(c, fld), 0, field_count(c, fld) * (c->precision == PNP_FP64 ? 8 : 4), c->stream));
  for (int fld : {PNP_HCP, PNP_HCM}) CK(cudaMemsetAsync(field_ptr(c, fld), 0, field_count(c, fld) * 8, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->have_state = true;
  c->fp64_fresh = true;
  c->refs_valid = false;
  return PNP_OK;
}

int pnp_wall_labels(pnp_ctx* f, pnp_ctx* c, float* T) {
  if (!f || !c || !T || f == c) return PNP_ERR_ARG;
  if (!f->have_state) return PNP_ERR_STATE;
  int err = 0;
  const WallMap wm = wall_map(f, c, &err);
  if (err) return err;
  IonView iv{};
  int r = ion_view(f, &iv);
  if (r) return r;
  double* scr = f->stage + f->nv - 3 * (size_t)f->g.ny;   // ycf, dyf, hf
  std::vector<double> pack(3 * (size_t)f->g.ny, 0.0);
  for (int j = 0; j < f->g.nyc; ++j) { pack[j] = f->yc[j]; pack[f->g.ny + j] = f->dy[j]; }
  for (int j = 0; j < f->g.ny; ++j) pack[2 * f->g.ny + j] = f->h[j];
  CK(cudaMemcpyAsync(scr, pack.data(), sizeof(double) * pack.size(), cudaMemcpyHostToDevice, f->stream));
  const double h0c = c->h[0];
  cudaError_t e = f->precision == PNP_FP64
                      ? launch_wall_labels<double>((const double*)f->u, (const double*)f->v, (const double*)f->w, iv,
                                                   scr, scr + f->g.ny, scr + 2 * f->g.ny, wm, h0c, f->ph.V, f->ph.Uw,
                                                   f->ph.D, T, f->stream)
                      : launch_wall_labels<float>((const float*)f->u, (const float*)f->v, (const float*)f->w, iv, scr,
                                                  scr + f->g.ny, scr + 2 * f->g.ny, wm, h0c, f->ph.V, f->ph.Uw,
                                                  f->ph.D, T, f->stream);
  if (e != cudaSuccess) return PNP_ERR_CUDA;
  CK(cudaStreamSynchronize(f->stream));
  return PNP_OK;
}

namespace {
int set_wall_values(pnp_ctx* c, const float* X, int ncells, const float* Y, bool stress) {
  if (!c || (Y && (!X || ncells < 1 || ncells > 8))) return PNP_ERR_ARG;
  const size_t P = (size_t)c->g.nz * c->g.nx;
  const bool was = c->slip_on, was_stress = c->wall_stress;
  if (!Y) {
    c->slip_on = false;
    c->wall_stress = false;
  } else {
    const double h0b = c->h[0], h0t = c->h[c->g.nyc];
    cudaError_t e = c->precision == PNP_FP64
                        ? launch_set_slip<double>(X, ncells, Y, P, c->ph.Uw, h0b, h0t, (double*)c->wall_u,
                                                  (double*)c->wall_w, c->stream)
                        : launch_set_slip<float>(X, ncells, Y, P, c->ph.Uw, h0b, h0t, (float*)c->wall_u,
                                                 (float*)c->wall_w, c->stream);
    if (e != cudaSuccess) return PNP_ERR_CUDA;
    c->slip_on = true;
    c->wall_stress = stress;
  }
  if (was != c->slip_on || was_stress != c->wall_stress) drop_graph(c);
  return PNP_OK;
}
}  // namespace

int pnp_set_wall_slip(pnp_ctx* c, const float* X, int ncells, const float* Y) {
  return set_wall_values(c, X, ncells, Y, false);
}

int pnp_set_wall_stress(pnp_ctx* c, const float* X, int ncells, const float* Y) {
  return set_wall_values(c, X, ncells, Y, true);
}

int pnp_set_wallmodel_coupling(pnp_ctx* c, int mode, double relax) {
  if (!c || mode < 0 || mode > 3 || !(relax > 0.0) || relax > 1.0) return PNP_ERR_ARG;
  c->wm_mode = mode;
  c->wm_relax = (float)relax;
  c->wm_have_prev = false;
  return PNP_OK;
}

namespace {
// Lift of the offset map: the charge-free potential of wall offsets B, T kept
// with their plane means (relative to the uniform walls, so V and the constant
// offset stay those of pnp_set_params).
cudaError_t edl_lift(pnp_ctx* c) {
  const Metrics m = metrics(c);
  cplx<double>* spec = (cplx<double>*)c->spec;
  const cplx<double>* twx = (const cplx<double>*)c->twx_d;
  const cplx<double>* twp = (const cplx<double>*)c->twp_d;
  const cplx<double>* twz = (const cplx<double>*)c->twz_d;
  cudaError_t e = launch_wall_lift_source(c->sreal, c->wallB_d, c->wallT_d, 0.0, 0.0, c->yc_d, c->g, c->stream);
  if (e == cudaSuccess)
    e = launch_fft_x_fwd<double, double>(PoissonSrc::Plain, nullptr, nullptr, nullptr, nullptr, nullptr, c->sreal, 1.0,
                                         c->g, m, spec, twx, twp, c->stream);
  if (e == cudaSuccess) e = spectral_solve<double>(c, spec, twz, false);
  if (e == cudaSuccess)
    e = launch_fft_x_inv<double, double>(PoissonDst::Plain, spec, c->g, m, twx, twp, 0.0, c->lift64, c->stream);
  if (e == cudaSuccess)
    e = launch_wall_lift_finish(c->lift64, c->lift32, c->wallB_d, c->wallT_d, 0.0, 0.0, 0.0, c->yc_d, c->g, c->stream);
  return e;
}

int edl_potential(pnp_ctx* c, const float* X, int ncells, const float* Y) {
  if (!c->have_state) return PNP_ERR_STATE;
  const size_t P = (size_t)c->g.nz * c->g.nx;
  if (!c->edl_map) {
    if (c->wall_map) return PNP_ERR_UNSUPPORTED;   // the user's wall-potential map is set
    CK(cudaMemsetAsync(c->wallB_d, 0, sizeof(double) * P, c->stream));
    CK(cudaMemsetAsync(c->wallT_d, 0, sizeof(double) * P, c->stream));
    CK(cudaMemsetAsync(c->lift64, 0, sizeof(double) * c->nc, c->stream));   // no offsets yet: no lift
    CK(cudaMemsetAsync(c->lift32, 0, sizeof(float) * c->nc, c->stream));
    c->edl_map = true;
    c->wall_map = true;
    c->wall_off = 0.0;
    drop_graph(c);
  }
  const double lim = std::max(1.0, std::fabs(c->ph.V));
  CK(launch_edl_offsets(X, ncells, Y, P, c->edl_phi_gain, lim, c->lift64, c->g.nyc, c->wallB_d, c->wallT_d,
                        c->stream));
  CK(edl_lift(c));
  // the potential of the present ions under the moved walls: in a mixed context that
  // steps on its shadows, the step's own potential pipeline (writes phi')
  if (c->precision == PNP_MIXED && c->refs_valid) {
    CK(c->policy == PNP_POLICY_FP64_SOLVES ? potential_mixed_fp64(c, c->stream, c->spec, c->dscr)
                                           : potential_mixed(c, c->stream, c->spec, c->dscr));
    c->fp64_fresh = false;
    return PNP_OK;
  }
  int r = materialize(c);
  if (r) return r;
  CK(c->precision == PNP_FP64 ? potential_solve<double>(c) : potential_solve<float>(c));
  return PNP_OK;
}

int flux_fix(pnp_ctx* c, const float* Y, double dt) {
  if (!c->have_state) return PNP_ERR_STATE;
  IonView iv{};
  int r = ion_view(c, &iv);
  if (r) return r;
  const cudaError_t e =
      c->precision == PNP_FP64
          ? launch_wall_flux_fix<double>(iv, (const double*)c->v, c->idy_d, c->ih_d, c->g, c->ph.D, Y,
                                         c->edl_flux_gain, dt, c->stream)
          : launch_wall_flux_fix<float>(iv, (const float*)c->v, c->idy_d, c->ih_d, c->g, c->ph.D, Y, c->edl_flux_gain,
                                        dt, c->stream);
  if (!iv.cp) c->fp64_fresh = false;   // the shadows were updated, not the FP64 copies
  return e == cudaSuccess ? PNP_OK : PNP_ERR_CUDA;
}
}  // namespace

int pnp_set_wallmodel_edl(pnp_ctx* c, double potential_gain, double flux_gain) {
  if (!c || !(potential_gain >= 0.0 && potential_gain <= 1.0) || !(flux_gain >= 0.0 && flux_gain <= 1.0))
    return PNP_ERR_ARG;
  c->edl_phi_gain = potential_gain;
  c->edl_flux_gain = flux_gain;
  if (potential_gain == 0.0 && c->edl_map) {   // the uniform walls return
    c->edl_map = false;
    return pnp_set_wall_potential(c, nullptr, nullptr);
  }
  return PNP_OK;
}

int pnp_set_wall_edl(pnp_ctx* c, const float* X, int ncells, const float* Y) {
  if (!c || !X || !Y || ncells < 1 || ncells > 8 || ncells > c->g.nyc || !(c->edl_phi_gain > 0.0))
    return PNP_ERR_ARG;
  return edl_potential(c, X, ncells, Y);
}

int pnp_correct_wall_flux(pnp_ctx* c, const float* Y, double dt) {
  if (!c || !Y || !(dt > 0.0) || !(c->edl_flux_gain > 0.0) || c->g.nyc < 4) return PNP_ERR_ARG;
  return flux_fix(c, Y, dt);
}

int pnp_step_wallmodel(pnp_ctx* c, pnp_mlp* m, int nsteps, double dt) {
  if (!c || !m || nsteps < 0) return PNP_ERR_ARG;
  const int rows = 2 * c->g.nz * c->g.nx;
  if (rows > m->max_batch) return PNP_ERR_ARG;
  if (c->edl_flux_gain > 0.0 && c->g.nyc < 4) return PNP_ERR_ARG;
  for (int n = 0; n < nsteps; ++n) {
    int r = pnp_wall_features(c, 8, c->featX);
    if (r) return r;
    CK(mlp_forward(m->b, c->featX, rows, c->featY, c->stream));
    if (c->wm_mode == 2) CK(launch_mean_rates(c->featY, rows / 2, c->stream));
    if (c->wm_mode <= 2) {   // mode 3 leaves the wall shear to the solver's own no-slip walls
      if (c->wm_relax < 1.f) {   // the rates used move a fraction of the way to the prediction
        CK(launch_relax_rates(c->featY, c->featYprev, rows, c->wm_have_prev ? c->wm_relax : 1.f, c->stream));
        c->wm_have_prev = true;
      }
      r = set_wall_values(c, c->featX, 8, c->featY, c->wm_mode >= 1);
      if (r) return r;
    } else if (c->slip_on) {
      r = set_wall_values(c, nullptr, 0, nullptr, false);
      if (r) return r;
    }
    if (c->edl_phi_gain > 0.0) {
      r = edl_potential(c, c->featX, 8, c->featY);
      if (r) return r;
    }
    r = pnp_step(c, 1, dt);
    if (r) return r;
    if (c->edl_flux_gain > 0.0) {
      r = flux_fix(c, c->featY, dt);
      if (r) return r;
    }
  }
  return PNP_OK;
}

const char* pnp_error_string(int code) {
  switch (code) {
    case PNP_OK: return "ok";
    case PNP_ERR_ARG: return "invalid argument";
    case PNP_ERR_GRID: return "invalid grid (Nx, Nz powers of two in [4, 4096]; Ny >= 3; increasing y faces)";
    case PNP_ERR_WORKSPACE: return "workspace too small or not 256-byte aligned";
    case PNP_ERR_CUDA: return "CUDA runtime error";
    case PNP_ERR_STATE: return "parameters or state not set";
    case PNP_ERR_NONFINITE: return "non-finite value in a prognostic field";
    case PNP_ERR_NEGATIVE_C: return "negative ion concentration";
    case PNP_ERR_UNSUPPORTED: return "unsupported option";
    case PNP_ERR_TIMEOUT: return "an asynchronous copy did not complete within the kernel's wait limit";
    case PNP_ERR_TOO_LARGE: return "grid exceeds the static scratch of pnp_poisson_noalloc (2^20 spectral points)";
    case PNP_ERR_CFL: return "advective CFL number of the last step above its limit";
    case PNP_ERR_DPHI: return "potential step between neighbouring cells above its limit";
    default: return "unknown error";
  }
}

void pnp_destroy(pnp_ctx* c) {
  if (!c) return;
  drop_graph(c);
  if (c->aux) {
    cudaStreamSynchronize(c->aux);
    cudaStreamDestroy(c->aux);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  delete c;
}

}  // extern "C"
