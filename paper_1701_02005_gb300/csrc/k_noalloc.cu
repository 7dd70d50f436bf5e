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
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "pnp_common.cuh"

using namespace pnp;

namespace {

// Maximum sizes served by the static scratch.
constexpr size_t kNaMaxSpec = (size_t)1 << 20;   // spectral points (Ny-1) * Nz * pitch(Nx/2+1)
constexpr int kNaMaxNy = 2049;                   // y face nodes (the faces travel as a kernel argument)
constexpr int kNaMaxN = 4096;                    // Nx and Nz

// Layout of the scratch, in doubles; every block starts on a 256-byte boundary.
constexpr size_t al32(size_t n) { return (n + 31) / 32 * 32; }
constexpr size_t kOffSpec = 0;                                      // complex<double> [kNaMaxSpec]
constexpr size_t kOffDscr = kOffSpec + 2 * kNaMaxSpec;              // complex<double> [kNaMaxSpec]
constexpr size_t kOffCpr = kOffDscr + 2 * kNaMaxSpec;               // double [kNaMaxSpec]
constexpr size_t kOffInv = kOffCpr + kNaMaxSpec;                    // double [kNaMaxSpec]
constexpr size_t kOffConst = kOffInv + kNaMaxSpec;                  // grid constants below
constexpr size_t kConstRows = al32(3 * (size_t)kNaMaxNy);           // a, b, c of the y-operator
constexpr size_t kConstKx = al32(kNaMaxN / 2 + 8);                  // kx2 (padded pitch)
constexpr size_t kConstKz = al32(kNaMaxN);                          // kz2
constexpr size_t kConstTwx = al32(2 * (kNaMaxN / 2));               // complex exp(-2 pi i t / (Nx/2))
constexpr size_t kConstTwp = al32(2 * (kNaMaxN / 2 + 1));           // complex exp(-2 pi i t / Nx)
constexpr size_t kConstTwz = al32(2 * kNaMaxN);                     // complex exp(-2 pi i t / Nz)
constexpr size_t kConstTotal = kConstRows + kConstKx + kConstKz + kConstTwx + kConstTwp + kConstTwz;
constexpr size_t kScratchDoubles = kOffConst + kConstTotal;         // ~48.3 MB

// The y faces passed by value: a kernel argument is copied when the launch is
// issued, so no host buffer has to outlive the call (16,392 bytes, inside the
// 32,764-byte parameter limit).
struct NaFaces {
  double y[kNaMaxNy];
};

}  // namespace

static __device__ __align__(256) double g_poisson_scratch[kScratchDoubles];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;   // guards the per-device addresses below
double* g_scratch_ptr[kMaxDevices] = {nullptr};

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

// Grid constants of one solve, written into the scratch in stream order (so a
// later call on the same stream cannot overwrite them while this one runs):
// the rows (a, b, c) of the finite-volume second difference in y (walls at
// the first and last face, forced to -1 and +1; Dirichlet: the wall value
// sits on the wall face, Neumann: no flux through it), the modified
// wavenumbers (2 - 2 cos(2 pi m / N)) / d^2, and the twiddles of the real
// x-transform and the complex z-transform.  Every entry the solve reads is
// written, padding included.
__global__ void k_na_constants(NaFaces f, int ny, int nx, int nz, double dx, double dz, int dirichlet,
                               double* __restrict__ cst) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nyc = ny - 1, mh = nx / 2 + 1, mp = (mh + 7) / 8 * 8, Lh = nx / 2;
  double* rows = cst;
  double* kx2 = rows + kConstRows;
  double* kz2 = kx2 + kConstKx;
  double* twx = kz2 + kConstKz;
  double* twp = twx + kConstTwx;
  double* twz = twp + kConstTwp;
  auto face = [&](int j) { return j == 0 ? -1.0 : (j == ny - 1 ? 1.0 : f.y[j]); };
  auto centre = [&](int j) { return 0.5 * (face(j) + face(j + 1)); };
  if (t < nyc) {
    const double dyj = face(t + 1) - face(t);
    const double hlo = t == 0 ? 0.5 * dyj : centre(t) - centre(t - 1);
    const double hhi = t == nyc - 1 ? 0.5 * dyj : centre(t + 1) - centre(t);
    const double lo = 1.0 / (hlo * dyj), hi = 1.0 / (hhi * dyj);
    double a = 0.0, b = 0.0, c = 0.0;
    if (t > 0) { a = lo; b -= lo; }
    else if (dirichlet) b -= lo;
    if (t < nyc - 1) { c = hi; b -= hi; }
    else if (dirichlet) b -= hi;
    rows[t] = a;
    rows[ny + t] = b;
    rows[2 * ny + t] = c;
  }
  if (t < mp) kx2[t] = t < mh ? (2.0 - 2.0 * cospi(2.0 * t / nx)) / (dx * dx) : 0.0;
  if (t < nz) kz2[t] = (2.0 - 2.0 * cospi(2.0 * t / nz)) / (dz * dz);
  double sn, cs;
  if (t < Lh) { sincospi(2.0 * t / Lh, &sn, &cs); twx[2 * t] = cs; twx[2 * t + 1] = -sn; }
  if (t <= Lh) { sincospi(2.0 * t / nx, &sn, &cs); twp[2 * t] = cs; twp[2 * t + 1] = -sn; }
  if (t < nz) { sincospi(2.0 * t / nz, &sn, &cs); twz[2 * t] = cs; twz[2 * t + 1] = -sn; }
}

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
  // the faces must increase; the walls are taken as -1 and +1
  for (int j = 0; j < ny - 1; ++j) {
    const double y0 = j == 0 ? -1.0 : y_faces_host[j];
    const double y1 = j + 1 == ny - 1 ? 1.0 : y_faces_host[j + 1];
    if (!(y1 - y0 > 0.0)) return PNP_ERR_GRID;
  }
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_setup_mutex);
    int r = scratch_address(&base);
    if (r) return r;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const bool dir = bc == PNP_DIRICHLET;
  const double dx = Lx / nx, dz = Lz / nz;
  double* dconst = base + kOffConst;
  NaFaces faces;
  std::memset(&faces, 0, sizeof(faces));
  std::memcpy(faces.y, y_faces_host, sizeof(double) * (size_t)ny);
  {
    const int need = std::max(std::max(nyc, mp), std::max(nz, nx / 2 + 1));
    k_na_constants<<<(need + 127) / 128, 128, 0, s>>>(faces, ny, nx, nz, dx, dz, dir ? 1 : 0, dconst);
    if (cudaGetLastError() != cudaSuccess) return PNP_ERR_CUDA;
  }

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
