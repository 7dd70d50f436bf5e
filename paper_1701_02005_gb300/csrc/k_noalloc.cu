// pnp_poisson_noalloc: the separable Poisson solve of pnp_poisson for callers
// that cannot allocate device memory.
//
// pnp_poisson needs a context, and a context needs a device workspace that the
// caller allocates.  Some callers cannot do that: code embedded in a host
// application or framework that owns every device allocation and forbids its
// plug-ins to call cudaMalloc, or code on a latency-critical path where an
// allocation (which may synchronise the device or fail under memory pressure)
// is not acceptable.  This entry point needs no context and allocates nothing:
// its scratch (spectral buffer, elimination factors, FP64 sweep values, grid
// rows, wavenumbers, FFT tables) is one file-scope static device array of
// fixed size, which every GPU that loads the library holds until the process
// exits.  The caller still passes the right-hand side and the solution array.
#include <cmath>
#include <cstring>
#include <mutex>

#include "pnp_common.cuh"

using namespace pnp;

namespace {

// Maximum sizes served by the static scratch.
constexpr size_t kNaMaxSpec = (size_t)1 << 20;   // spectral points (Ny-1) * Nz * pitch(Nx/2+1)
constexpr int kNaMaxNy = 4097;                   // y face nodes
constexpr int kNaMaxN = 4096;                    // Nx and Nz

// Layout of the scratch, in doubles; every block starts on a 256-byte boundary.
constexpr size_t al32(size_t n) { return (n + 31) / 32 * 32; }
constexpr size_t kOffSpec = 0;                                      // complex<double> [kNaMaxSpec]
constexpr size_t kOffDscr = kOffSpec + 2 * kNaMaxSpec;              // complex<double> [kNaMaxSpec]
constexpr size_t kOffCpr = kOffDscr + 2 * kNaMaxSpec;               // double [kNaMaxSpec]
constexpr size_t kOffInv = kOffCpr + kNaMaxSpec;                    // double [kNaMaxSpec]
constexpr size_t kOffConst = kOffInv + kNaMaxSpec;                  // host-computed constants below
constexpr size_t kConstRows = al32(3 * (size_t)kNaMaxNy);           // a, b, c of the y-operator
constexpr size_t kConstKx = al32(kNaMaxN / 2 + 8);                  // kx2 (padded pitch)
constexpr size_t kConstKz = al32(kNaMaxN);                          // kz2
constexpr size_t kConstTwx = al32(2 * (kNaMaxN / 2));               // complex exp(-2 pi i t / (Nx/2))
constexpr size_t kConstTwp = al32(2 * (kNaMaxN / 2 + 1));           // complex exp(-2 pi i t / Nx)
constexpr size_t kConstTwz = al32(2 * kNaMaxN);                     // complex exp(-2 pi i t / Nz)
constexpr size_t kConstTotal = kConstRows + kConstKx + kConstKz + kConstTwx + kConstTwp + kConstTwz;
constexpr size_t kScratchDoubles = kOffConst + kConstTotal;         // ~48.3 MB

}  // namespace

static __device__ __align__(256) double g_poisson_scratch[kScratchDoubles];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;   // guards the per-device addresses and the static host buffers below
double* g_scratch_ptr[kMaxDevices] = {nullptr};
// host-side work buffers (static, so that the call allocates no host memory either)
double g_host_const[kConstTotal];
double g_host_dy[kNaMaxNy], g_host_yc[kNaMaxNy], g_host_h[kNaMaxNy];

// Device address of the static scratch for the current device (looked up once
// per device; the name g_poisson_scratch is only a host-side stand-in).
// Call with g_setup_mutex held.
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PNP_ERR_CUDA;
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_poisson_scratch) != cudaSuccess || p == nullptr) return PNP_ERR_CUDA;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return PNP_OK;
}

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

}  // namespace

extern "C" int pnp_poisson_noalloc(int nx, int ny, int nz, double Lx, double Lz, const double* y_faces_host, int bc,
                                   const double* rhs_dev, double* x_dev, void* cuda_stream) {
  if (!y_faces_host || !rhs_dev || !x_dev || (bc != PNP_NEUMANN && bc != PNP_DIRICHLET) || !(Lx > 0) || !(Lz > 0))
    return PNP_ERR_ARG;
  if (!pow2(nx) || !pow2(nz) || nx < 4 || nz < 4 || ny < 3) return PNP_ERR_GRID;
  const int nyc = ny - 1;
  const int mh = nx / 2 + 1;
  const int mp = (mh + 7) / 8 * 8;
  const size_t nspec = (size_t)nyc * nz * mp;
  if (nx > kNaMaxN || nz > kNaMaxN || ny > kNaMaxNy || nspec > kNaMaxSpec) return PNP_ERR_TOO_LARGE;
  std::lock_guard<std::mutex> lk(g_setup_mutex);
  double* base = nullptr;
  int r = scratch_address(&base);
  if (r) return r;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // grid metrics from the y faces (the same finite-volume definitions as pnp_init_grid)
  double* dy = g_host_dy;
  double* yc = g_host_yc;
  double* h = g_host_h;
  for (int j = 0; j < nyc; ++j) {
    const double y0 = j == 0 ? -1.0 : y_faces_host[j];
    const double y1 = j + 1 == ny - 1 ? 1.0 : y_faces_host[j + 1];
    dy[j] = y1 - y0;
    yc[j] = 0.5 * (y0 + y1);
    if (!(dy[j] > 0.0)) return PNP_ERR_GRID;
  }
  h[0] = 0.5 * dy[0];
  for (int j = 1; j < nyc; ++j) h[j] = yc[j] - yc[j - 1];
  h[nyc] = 0.5 * dy[nyc - 1];
  // host-computed constants, packed as in the scratch layout
  double* cst = g_host_const;
  std::memset(cst, 0, sizeof(g_host_const));
  double* rows = cst;
  double* kx2 = rows + kConstRows;
  double* kz2 = kx2 + kConstKx;
  double* twx = kz2 + kConstKz;
  double* twp = twx + kConstTwx;
  double* twz = twp + kConstTwp;
  const bool dir = bc == PNP_DIRICHLET;
  for (int j = 0; j < nyc; ++j) {
    const double lo = 1.0 / (h[j] * dy[j]);
    const double hi = 1.0 / (h[j + 1] * dy[j]);
    double b = 0.0;
    if (j > 0) { rows[j] = lo; b -= lo; }
    else if (dir) b -= lo;
    if (j < nyc - 1) { rows[2 * ny + j] = hi; b -= hi; }
    else if (dir) b -= hi;
    rows[ny + j] = b;
  }
  const double dx = Lx / nx, dz = Lz / nz;
  for (int m = 0; m < mh; ++m) kx2[m] = (2.0 - 2.0 * std::cos(2.0 * M_PI * m / nx)) / (dx * dx);
  for (int n = 0; n < nz; ++n) kz2[n] = (2.0 - 2.0 * std::cos(2.0 * M_PI * n / nz)) / (dz * dz);
  const int Lh = nx / 2;
  for (int t = 0; t < Lh; ++t) { twx[2 * t] = std::cos(2.0 * M_PI * t / Lh); twx[2 * t + 1] = -std::sin(2.0 * M_PI * t / Lh); }
  for (int t = 0; t <= Lh; ++t) { twp[2 * t] = std::cos(2.0 * M_PI * t / nx); twp[2 * t + 1] = -std::sin(2.0 * M_PI * t / nx); }
  for (int t = 0; t < nz; ++t) { twz[2 * t] = std::cos(2.0 * M_PI * t / nz); twz[2 * t + 1] = -std::sin(2.0 * M_PI * t / nz); }
  double* dconst = base + kOffConst;
  // a pageable source is staged before cudaMemcpyAsync returns, so the static
  // host buffer may be reused by the next call as soon as this one returns
  if (cudaMemcpyAsync(dconst, cst, sizeof(g_host_const), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return PNP_ERR_CUDA;

  Geo g{};
  g.nx = nx; g.nz = nz; g.nyc = nyc; g.ny = ny; g.mh = mh; g.mp = mp;
  g.dx = dx; g.dz = dz; g.idx = 1.0 / dx; g.idz = 1.0 / dz;
  const Metrics m{};
  const YRows yr{dconst, dconst + ny, dconst + 2 * ny};
  cplx<double>* spec = reinterpret_cast<cplx<double>*>(base + kOffSpec);
  cplx<double>* dscr = reinterpret_cast<cplx<double>*>(base + kOffDscr);
  double* cpr = base + kOffCpr;
  double* inv = base + kOffInv;
  const double* dkx = dconst + kConstRows;
  const double* dkz = dkx + kConstKx;
  const cplx<double>* tx = reinterpret_cast<const cplx<double>*>(dkz + kConstKz);
  const cplx<double>* tp = reinterpret_cast<const cplx<double>*>(dkz + kConstKz + kConstTwx);
  const cplx<double>* tz = reinterpret_cast<const cplx<double>*>(dkz + kConstKz + kConstTwx + kConstTwp);
  // every scratch value read below is written earlier in this same call: nothing needs clearing
  if (launch_spec_factors(cpr, inv, dkx, dkz, yr, g, !dir, s) != cudaSuccess) return PNP_ERR_CUDA;
  if (launch_fft_x_fwd<double, double>(PoissonSrc::Plain, nullptr, nullptr, nullptr, nullptr, nullptr, rhs_dev, 1.0,
                                       g, m, spec, tx, tp, s) != cudaSuccess)
    return PNP_ERR_CUDA;
  if (launch_fft_z<double>(spec, tz, g, false, s) != cudaSuccess) return PNP_ERR_CUDA;
  const double scale = 1.0 / ((double)nx * (double)nz);
  if (launch_spec_thomas<double>(spec, dscr, cpr, inv, yr, g, scale, !dir, s) != cudaSuccess) return PNP_ERR_CUDA;
  if (launch_fft_z<double>(spec, tz, g, true, s) != cudaSuccess) return PNP_ERR_CUDA;
  if (launch_fft_x_inv<double, double>(PoissonDst::Plain, spec, g, m, tx, tp, 0.0, x_dev, s) != cudaSuccess)
    return PNP_ERR_CUDA;
  return PNP_OK;
}
