// Linear solves of the fractional step (arXiv:1701.02005, Numerical methods):
//  * wall-normal Crank-Nicolson solves (Thomas) for u, v, w and c+- ;
//  * the separable Poisson solver of the potential paragraph: real FFT in x,
//    complex FFT in z, one Thomas solve in y per wavenumber pair, inverse
//    FFTs; used for the pressure correction (Neumann) and the potential
//    perturbation phi (Dirichlet);
//  * the projection u = u_hat - alp dt grad(Phi_p), p += Phi_p.
//
// FFTs are radix-2 Stockham autosort transforms in shared memory (Stockham
// 1966; the formulation of Govindaraju et al., SC 2008).  A length-N real row
// is transformed as a length-N/2 complex sequence z_t = x_2t + i x_2t+1 and
// split into the N/2 + 1 non-negative frequencies.  Forward transforms carry
// no normalisation; the spectral solve multiplies by 1/(Nx Nz).
#include <type_traits>

#include "pnp_common.cuh"
#include "pnp_df.cuh"
#include "pnp_regfft.cuh"

namespace pnp {

// ---------------------------------------------------------------------------
// Crank-Nicolson y-solves.  One thread per (i, k) line; lines are consecutive
// in x so every plane access is coalesced.  The matrix I - s L_y is the same
// for every line, so its elimination factors (a, c, m) come precomputed.
// ---------------------------------------------------------------------------
template <typename TQ, typename TR>
__global__ void k_cn_thomas(TQ* __restrict__ q0, TR* __restrict__ r0, TQ* __restrict__ q1,
                            TR* __restrict__ r1, TQ* __restrict__ q2, TR* __restrict__ r2,
                            CNRows rows0, CNRows rows1, CNRows rows2, int n0, int n1, int n2,
                            int j00, int j01, int j02, size_t P) {
  constexpr int CH = 8;   // planes loaded ahead per sweep step
  const size_t line = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= P) return;
  TQ* q;
  TR* r;
  CNRows rw;
  int n, j0;
  if (blockIdx.y == 0) { q = q0; r = r0; rw = rows0; n = n0; j0 = j00; }
  else if (blockIdx.y == 1) { q = q1; r = r1; rw = rows1; n = n1; j0 = j01; }
  else { q = q2; r = r2; rw = rows2; n = n2; j0 = j02; }
  TR* rl = r + (size_t)j0 * P + line;
  TQ* ql = q + (size_t)j0 * P + line;
  double d = 0.0;
  for (int jb = 0; jb < n; jb += CH) {
    double rr[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u)
      if (jb + u < n) rr[u] = (double)rl[(size_t)(jb + u) * P];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int j = jb + u;
      if (j < n) {
        d = (rr[u] - rw.a[j] * d) * rw.m[j];
        rl[(size_t)j * P] = (TR)d;
      }
    }
  }
  double x = 0.0;
  for (int jb = n - 1; jb >= 0; jb -= CH) {
    double dd[CH], qq[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u)
      if (jb - u >= 0) {
        dd[u] = (double)rl[(size_t)(jb - u) * P];
        qq[u] = (double)ql[(size_t)(jb - u) * P];
      }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int j = jb - u;
      if (j >= 0) {
        x = dd[u] - rw.c[j] * x;
        ql[(size_t)j * P] = (TQ)(qq[u] + x);
      }
    }
  }
}

template <typename TV>
cudaError_t launch_cn_solves(const Fields<TV>& f, const Geo& g, const CNRows& vel, const CNRows& face,
                             const CNRows& ion, cudaStream_t s) {
  const size_t P = (size_t)g.nz * g.nx;
  const int T = g.lc_cn ? g.lc_cn : 128;
  dim3 grd((unsigned)((P + T - 1) / T), 3, 1);
  // u, w: nyc cells from plane 0; v: the nyc-1 interior faces from plane 1
  k_cn_thomas<TV, TV><<<grd, T, 0, s>>>(f.u, f.ru, f.v, f.rv, f.w, f.rw, vel, face, vel, g.nyc,
                                        g.nyc - 1, g.nyc, 0, 1, 0, P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 grd2((unsigned)((P + T - 1) / T), 2, 1);
  k_cn_thomas<double, double><<<grd2, T, 0, s>>>(f.cp, f.rcp, f.cm, f.rcm, f.cm, f.rcm, ion, ion, ion,
                                                 g.nyc, g.nyc, g.nyc, 0, 0, 0, P);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Shared-memory Stockham FFT of one sequence of length N (power of two)
// between buffers x and y: radix-4 stages, preceded by one radix-2 stage when
// log2 N is odd.  nt threads cooperate, this one is t0; tw[t] = exp(-2 pi i
// t / N).  Returns the buffer that holds the result.  Every thread of the
// block must call it (it synchronises the block).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ cplx<T> mul_i(cplx<T> z, bool neg) {   // +i z, or -i z when neg
  return neg ? cplx<T>{z.y, -z.x} : cplx<T>{-z.y, z.x};
}

template <typename T>
__device__ cplx<T>* stockham(cplx<T>* x, cplx<T>* y, int N, const cplx<T>* __restrict__ tw, bool inverse,
                             int t0, int nt) {
  int Ns = 1;
  if ((__ffs(N) - 1) & 1) {
    const int half = N >> 1;
    for (int jj = t0; jj < half; jj += nt) {
      const cplx<T> a0 = x[jj], a1 = x[jj + half];
      y[2 * jj] = cadd(a0, a1);
      y[2 * jj + 1] = csub(a0, a1);
    }
    __syncthreads();
    cplx<T>* t = x;
    x = y;
    y = t;
    Ns = 2;
  }
  const int q = N >> 2;
  for (; Ns < N; Ns <<= 2) {
    const int tstride = N / (Ns * 4);
    for (int jj = t0; jj < q; jj += nt) {
      const int k = jj & (Ns - 1);
      cplx<T> a = x[jj], b = x[jj + q], c = x[jj + 2 * q], d = x[jj + 3 * q];
      if (k != 0) {
        cplx<T> w1 = tw[k * tstride], w2 = tw[2 * k * tstride], w3 = tw[3 * k * tstride];
        if (inverse) { w1.y = -w1.y; w2.y = -w2.y; w3.y = -w3.y; }
        b = cmul(b, w1);
        c = cmul(c, w2);
        d = cmul(d, w3);
      }
      const cplx<T> apc = cadd(a, c), amc = csub(a, c), bpd = cadd(b, d), bmd = csub(b, d);
      const cplx<T> ib = mul_i(bmd, !inverse);   // forward: -i (b - d); inverse: +i (b - d)
      const int dst = ((jj - k) << 2) + k;
      y[dst] = cadd(apc, bpd);
      y[dst + Ns] = cadd(amc, ib);
      y[dst + 2 * Ns] = csub(apc, bpd);
      y[dst + 3 * Ns] = csub(amc, ib);
    }
    __syncthreads();
    cplx<T>* t = x;
    x = y;
    y = t;
  }
  return x;
}

// Source of the forward x-transform: one real value at (j, k, i).
template <typename T, typename TV>
struct SrcArgs {
  PoissonSrc kind;
  const TV *u, *v, *w;
  const double *cp, *cm;
  const T* plain;
  double scale;
  const float *sa, *sb;   // FP32 charge shadows c+', c-'
  T sx, sz;               // scale / dx, scale / dz in the transform's precision
  const T* idyT;          // 1 / dy in the transform's precision
  T ss;                   // scale
  const float *la, *lb;   // low parts of the double-float ion fluctuations (ChargeShadowDF)
};

template <typename T, typename TV>
__device__ __forceinline__ T src_value(const SrcArgs<T, TV>& a, const Geo& g, const Metrics& m, int j,
                                       int k, int i) {
  const size_t c = cidx(j, k, i, g.nz, g.nx);
  if (a.kind == PoissonSrc::Divergence) {
    // div(u_hat) / (alp dt): finite-volume form of Eq. (2)
    const int ip = (i + 1 == g.nx) ? 0 : i + 1;
    const int kp = (k + 1 == g.nz) ? 0 : k + 1;
    const T du = ((T)a.u[cidx(j, k, ip, g.nz, g.nx)] - (T)a.u[c]) * a.sx;
    const T dv = ((T)a.v[c + (size_t)g.nz * g.nx] - (T)a.v[c]) * (a.idyT[j] * a.ss);
    const T dw = ((T)a.w[cidx(j, kp, i, g.nz, g.nx)] - (T)a.w[c]) * a.sz;
    return du + dv + dw;
  } else if (a.kind == PoissonSrc::Charge) {
    // Eq. (4): -(c+ - c-) / (2 lam^2)
    return (T)(-(a.cp[c] - a.cm[c]) * a.scale);
  } else if (a.kind == PoissonSrc::ChargeShadow) {
    // fluctuating charge about the reference profile, FP32
    return T(-(a.sa[c] - a.sb[c])) * a.ss;
  } else if (a.kind == PoissonSrc::ChargeShadowDF) {
    // the same from the full double-float fluctuations (S + L), in T
    return -(((T)a.sa[c] + (T)a.la[c]) - ((T)a.sb[c] + (T)a.lb[c])) * a.ss;
  }
  return a.plain[c];
}

// Forward x-transform of rows (j, k): blockDim = (TX, RY); one row per threadIdx.y.
template <typename T, typename TV>
__global__ void k_fft_x_fwd(SrcArgs<T, TV> src, Geo g, Metrics m, cplx<T>* __restrict__ spec,
                            const cplx<T>* __restrict__ tw_half, const cplx<T>* __restrict__ tw_post) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* sm = reinterpret_cast<cplx<T>*>(smem_raw);
  const int Lh = g.nx >> 1;
  const int nrows = g.nyc * g.nz;
  const int row = blockIdx.x * blockDim.y + threadIdx.y;
  cplx<T>* xa = sm + (size_t)threadIdx.y * 2 * Lh;
  cplx<T>* xb = xa + Lh;
  const bool live = row < nrows;
  const int j = live ? row / g.nz : 0, k = live ? row % g.nz : 0;
  for (int t = threadIdx.x; t < Lh; t += blockDim.x) {
    cplx<T> z = {T(0), T(0)};
    if (live) z = {src_value(src, g, m, j, k, 2 * t), src_value(src, g, m, j, k, 2 * t + 1)};
    xa[t] = z;
  }
  __syncthreads();
  cplx<T>* Z = stockham(xa, xb, Lh, tw_half, false, threadIdx.x, blockDim.x);
  if (!live) return;
  cplx<T>* out = spec + (size_t)row * g.mp;
  for (int mm = threadIdx.x; mm <= Lh; mm += blockDim.x) {
    const cplx<T> zm = Z[mm == Lh ? 0 : mm];
    const cplx<T> zc = cconj(Z[(Lh - mm) == Lh ? 0 : (Lh - mm)]);
    const cplx<T> E = {T(0.5) * (zm.x + zc.x), T(0.5) * (zm.y + zc.y)};
    const cplx<T> dd = csub(zm, zc);
    const cplx<T> O = {T(0.5) * dd.y, T(-0.5) * dd.x};   // (zm - zc) / (2i)
    out[mm] = cadd(E, cmul(tw_post[mm], O));
  }
}

// Row buffer of the register x-transforms: the exchange is laid out
// [k1][g] with a stride of G + 1 (so the G-point reads of pass 2, one run of G
// values per thread, fall in distinct banks), the natural-order row reuses it,
// and the row stride is 8 mod 16 complex values so that the two rows served
// by one half-warp of 64-bit accesses use opposite halves of the banks.
template <int NH, int R1>
constexpr int fx_row_stride() {
  constexpr int G = NH / R1;
  constexpr int need = R1 * (G + 1) > NH + 1 ? R1 * (G + 1) : NH + 1;
  return need + ((8 - need % 16) + 16) % 16;
}

// Two consecutive values p[0], p[1] (p 8-byte aligned for FP32, 16-byte for
// FP64) as one vector load, converted to T.
template <typename T, typename S>
__device__ __forceinline__ cplx<T> ld_pair(const S* p) {
  if constexpr (sizeof(S) == sizeof(float)) {
    const float2 a = *reinterpret_cast<const float2*>(p);
    return {(T)a.x, (T)a.y};
  } else {
    const double2 a = *reinterpret_cast<const double2*>(p);
    return {(T)a.x, (T)a.y};
  }
}

// Real x-transforms (FP32 or FP64) with the two-pass register FFT (pnp_regfft.cuh) of
// the half-length complex sequence z_t = x_2t + i x_2t+1.  G = NH / R1 threads
// own a row (consecutive lanes of one warp, so every exchange inside a row
// needs only a warp barrier); ROWS rows per block.
//
// Forward: thread g forms z_t for t = g + G r from the source, does the
// R1-point DFT, twiddles, exchanges, does its G-point DFTs, writes Z to the
// row buffer in natural order, and the row's threads split the real-FFT
// post-processing X_m = E_m + W_N^m O_m over m = 0 .. NH.
template <int NH, int R1, typename T, typename TV>
__global__ void __launch_bounds__(256) k_fft_x_fwd_reg(SrcArgs<T, TV> src, Geo g, Metrics mt,
                                                       cplx<T>* __restrict__ spec,
                                                       const cplx<T>* __restrict__ tw_half,
                                                       const cplx<T>* __restrict__ tw_post) {
  constexpr int G = NH / R1, PER = R1 / G;
  static_assert(R1 % G == 0 && 32 % G == 0, "row of whole transforms inside one warp");
  extern __shared__ __align__(16) unsigned char fx_smem[];
  cplx<T>* twh = reinterpret_cast<cplx<T>*>(fx_smem);   // [NH]
  cplx<T>* twp = twh + NH;                               // [NH + 1]
  cplx<T>* rows = twp + NH + 1;                          // [ROWS][row stride]
  const int gi = threadIdx.x, ry = threadIdx.y, tid = ry * G + gi;
  const int nthr = G * blockDim.y;
  for (int e = tid; e < NH; e += nthr) twh[e] = tw_half[e];
  for (int e = tid; e <= NH; e += nthr) twp[e] = tw_post[e];
  const int nrows = g.nyc * g.nz;
  const int row = blockIdx.x * blockDim.y + ry;
  const bool live = row < nrows;
  const int j = live ? row / g.nz : 0, k = live ? row % g.nz : 0;
  cplx<T> v[R1];
  const size_t rbase = ((size_t)j * g.nz + k) * g.nx;   // this row's first cell
  if (live && src.kind == PoissonSrc::Divergence) {
    // both samples of z_t from paired loads: x-faces 2t, 2t+1, 2t+2 (periodic),
    // v on the faces below / above, w on the z-faces k, k+1
    const size_t P = (size_t)g.nz * g.nx;
    const int kp = (k + 1 == g.nz) ? 0 : k + 1;
    const size_t rbp = ((size_t)j * g.nz + kp) * g.nx;
    const T sy = src.idyT[j] * src.ss;
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      const int i = 2 * (gi + G * r);
      const cplx<T> u01 = ld_pair<T>(src.u + rbase + i);
      const T u2 = (T)src.u[rbase + (i + 2 == g.nx ? 0 : i + 2)];
      const cplx<T> vb = ld_pair<T>(src.v + rbase + i);
      const cplx<T> vt = ld_pair<T>(src.v + rbase + P + i);
      const cplx<T> wk = ld_pair<T>(src.w + rbase + i);
      const cplx<T> wkp = ld_pair<T>(src.w + rbp + i);
      v[r] = {(u01.y - u01.x) * src.sx + (vt.x - vb.x) * sy + (wkp.x - wk.x) * src.sz,
              (u2 - u01.y) * src.sx + (vt.y - vb.y) * sy + (wkp.y - wk.y) * src.sz};
    }
  } else if (live && src.kind == PoissonSrc::ChargeShadow) {
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      const int i = 2 * (gi + G * r);
      const cplx<T> a = ld_pair<T>(src.sa + rbase + i);
      const cplx<T> b = ld_pair<T>(src.sb + rbase + i);
      v[r] = {(-(a.x - b.x)) * src.ss, (-(a.y - b.y)) * src.ss};
    }
  } else {
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      const int t = gi + G * r;
      v[r] = live ? cplx<T>{src_value(src, g, mt, j, k, 2 * t), src_value(src, g, mt, j, k, 2 * t + 1)}
                  : cplx<T>{T(0), T(0)};
    }
  }
  __syncthreads();   // twiddle tables
  rfft::dft<false, R1>(v);
  cplx<T>* xr = rows + (size_t)ry * fx_row_stride<NH, R1>();
  rfft::static_for<0, R1>([&](auto kc) {
    constexpr int k1 = decltype(kc)::value;
    xr[k1 * (G + 1) + gi] = cmul(v[rfft::bitrev(k1, R1)], twh[gi * k1]);
  });
  __syncwarp();
  cplx<T> w[PER][G];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int k1 = gi * PER + p;
#pragma unroll
    for (int q = 0; q < G; ++q) w[p][q] = xr[k1 * (G + 1) + q];
    rfft::dft<false, G>(w[p]);
  }
  __syncwarp();
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int k1 = gi * PER + p;
    rfft::static_for<0, G>([&](auto kc) {
      constexpr int k2 = decltype(kc)::value;
      xr[k1 + R1 * k2] = w[p][rfft::bitrev(k2, G)];
    });
  }
  __syncwarp();
  if (!live) return;
  cplx<T>* out = spec + (size_t)row * g.mp;
  for (int mm = gi; mm <= NH; mm += G) {
    const cplx<T> zm = xr[mm == NH ? 0 : mm];
    const cplx<T> zc = cconj(xr[mm == 0 ? 0 : NH - mm]);
    const cplx<T> E = {T(0.5) * (zm.x + zc.x), T(0.5) * (zm.y + zc.y)};
    const cplx<T> dd = csub(zm, zc);
    const cplx<T> O = {T(0.5) * dd.y, T(-0.5) * dd.x};   // (zm - zc) / (2i)
    out[mm] = cadd(E, cmul(twp[mm], O));
  }
}

// n consecutive outputs (n = 2 or 4; out aligned to n elements) in vector stores.
template <typename TO, int N>
__device__ __forceinline__ void store_out(TO* out, const TO (&y)[N]) {
  if constexpr (sizeof(TO) == 4 && N == 4) {
    *reinterpret_cast<float4*>(out) = make_float4(y[0], y[1], y[2], y[3]);
  } else if constexpr (sizeof(TO) == 4 && N == 2) {
    *reinterpret_cast<float2*>(out) = make_float2(y[0], y[1]);
  } else {
#pragma unroll
    for (int q = 0; q < N; q += 2) *reinterpret_cast<double2*>(out + q) = make_double2(y[q], y[q + 1]);
  }
}

// Inverse: thread g forms the pre-processed z_t (from X_t and conj X_{NH-t})
// for t = g + G r straight from the spectrum, runs the inverse transform and
// writes x_2t, x_2t+1 of t = k1 + R1 k2.
template <int NH, int R1, typename T, typename TO>
__global__ void __launch_bounds__(256) k_fft_x_inv_reg(PoissonDst dst, const cplx<T>* __restrict__ spec, Geo g,
                                                       Metrics mt, const cplx<T>* __restrict__ tw_half,
                                                       const cplx<T>* __restrict__ tw_post, double V,
                                                       TO* __restrict__ out, const double* __restrict__ plane_add,
                                                       const TO* __restrict__ cell_add) {
  constexpr int G = NH / R1, PER = R1 / G;
  static_assert(R1 % G == 0 && 32 % G == 0, "row of whole transforms inside one warp");
  extern __shared__ __align__(16) unsigned char fx_smem[];
  cplx<T>* twh = reinterpret_cast<cplx<T>*>(fx_smem);   // [NH] (conjugated)
  cplx<T>* twp = twh + NH;                               // [NH]
  cplx<T>* rows = twp + NH;                              // [ROWS][row stride]
  const int gi = threadIdx.x, ry = threadIdx.y, tid = ry * G + gi;
  const int nthr = G * blockDim.y;
  for (int e = tid; e < NH; e += nthr) {
    const cplx<T> a = tw_half[e];
    twh[e] = {a.x, -a.y};
    twp[e] = tw_post[e];
  }
  const int nrows = g.nyc * g.nz;
  const int row = blockIdx.x * blockDim.y + ry;
  const bool live = row < nrows;
  const cplx<T>* in = spec + (size_t)(live ? row : 0) * g.mp;
  __syncthreads();   // twiddle tables
  cplx<T> v[R1];
#pragma unroll
  for (int r = 0; r < R1; ++r) {
    const int t = gi + G * r;
    cplx<T> z = {T(0), T(0)};
    if (live) {
      const cplx<T> Xm = in[t];
      const cplx<T> Xc = cconj(in[NH - t]);
      const cplx<T> sum = cadd(Xm, Xc);
      const cplx<T> dif = csub(Xm, Xc);
      const cplx<T> tt = cmul(cconj(twp[t]), dif);
      z = {sum.x - tt.y, sum.y + tt.x};   // sum + i * tt
    }
    v[r] = z;
  }
  rfft::dft<true, R1>(v);
  cplx<T>* xr = rows + (size_t)ry * fx_row_stride<NH, R1>();
  rfft::static_for<0, R1>([&](auto kc) {
    constexpr int k1 = decltype(kc)::value;
    xr[k1 * (G + 1) + gi] = cmul(v[rfft::bitrev(k1, R1)], twh[gi * k1]);
  });
  __syncwarp();
  if (!live) return;
  const int j = row / g.nz;
  const size_t base = (size_t)row * g.nx;
  const double add = dst == PoissonDst::Potential ? V * mt.yc[j] : 0.0;
  const T addT = dst == PoissonDst::PotentialShadow ? (T)plane_add[j] : T(0);
  // the thread's PER transforms first, so that the 2 PER consecutive outputs of
  // each k2 leave in one vector store (k1 = gi PER + p: pairs side by side)
  cplx<T> w[PER][G];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int k1 = gi * PER + p;
#pragma unroll
    for (int q = 0; q < G; ++q) w[p][q] = xr[k1 * (G + 1) + q];
    rfft::dft<true, G>(w[p]);
  }
  rfft::static_for<0, G>([&](auto kc) {
    constexpr int k2 = decltype(kc)::value;
    const size_t o = base + 2 * (size_t)(gi * PER + R1 * k2);
    TO y[2 * PER];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const cplx<T> z = w[p][rfft::bitrev(k2, G)];
      TO a0, a1;
      if (dst == PoissonDst::PotentialShadow) {
        a0 = (TO)(addT + z.x);
        a1 = (TO)(addT + z.y);
      } else if (dst == PoissonDst::Potential) {
        a0 = (TO)(add + (double)z.x);
        a1 = (TO)(add + (double)z.y);
      } else {
        a0 = (TO)z.x;
        a1 = (TO)z.y;
      }
      if (dst != PoissonDst::Plain && cell_add) {
        a0 += cell_add[o + 2 * p];
        a1 += cell_add[o + 2 * p + 1];
      }
      y[2 * p] = a0;
      y[2 * p + 1] = a1;
    }
    store_out<TO, 2 * PER>(out + o, y);
  });
}

// Rows per 128-thread block of the register x-transforms (smaller blocks share
// the GPU better with the other stream: 2.583 against 2.593 ms per step with
// 256 threads on the 256x193x256 workload), and shared memory.
template <int NH, int R1>
constexpr int fx_rows() { return 128 / (NH / R1); }
template <int NH, int R1, typename T>
constexpr size_t fx_smem() {
  return sizeof(cplx<T>) * ((size_t)2 * NH + 1 + (size_t)fx_rows<NH, R1>() * fx_row_stride<NH, R1>());
}

template <typename T>
static void fft_x_shape(const Geo& g, dim3& blk, dim3& grd, size_t& smem) {
  const int Lh = g.nx >> 1;
  int tx = Lh / 4 < 1 ? 1 : Lh / 4;
  if (tx > 128) tx = 128;
  int ry = 128 / tx;
  if (ry < 1) ry = 1;
  const int nrows = g.nyc * g.nz;
  blk = dim3(tx, ry, 1);
  grd = dim3((nrows + ry - 1) / ry, 1, 1);
  smem = (size_t)ry * 2 * Lh * sizeof(cplx<T>);
}

template <typename T, typename TV>
cudaError_t launch_fft_x_fwd(PoissonSrc kind, const TV* u, const TV* v, const TV* w, const double* cp,
                             const double* cm, const T* plain, double scale, const Geo& g,
                             const Metrics& m, cplx<T>* spec, const cplx<T>* tw_half,
                             const cplx<T>* tw_post, cudaStream_t s, const float* sa, const float* sb,
                             const T* idyT, const float* la, const float* lb) {
  SrcArgs<T, TV> a{kind, u, v, w, cp, cm, plain, scale, sa, sb, (T)(scale * g.idx), (T)(scale * g.idz), idyT,
                   (T)scale, la, lb};
  {
    auto go = [&](auto kern, int G, int rows, size_t smem) {
      if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
      }
      const int nrows = g.nyc * g.nz;
      kern<<<(nrows + rows - 1) / rows, dim3(G, rows), smem, s>>>(a, g, m, spec, tw_half, tw_post);
      return cudaGetLastError();
    };
    switch (g.nx / 2) {
      case 16: return go(k_fft_x_fwd_reg<16, 4, T, TV>, 4, fx_rows<16, 4>(), fx_smem<16, 4, T>());
      case 32: return go(k_fft_x_fwd_reg<32, 8, T, TV>, 4, fx_rows<32, 8>(), fx_smem<32, 8, T>());
      case 64: return go(k_fft_x_fwd_reg<64, 8, T, TV>, 8, fx_rows<64, 8>(), fx_smem<64, 8, T>());
      case 128: return go(k_fft_x_fwd_reg<128, 16, T, TV>, 8, fx_rows<128, 16>(), fx_smem<128, 16, T>());
      case 256: return go(k_fft_x_fwd_reg<256, 16, T, TV>, 16, fx_rows<256, 16>(), fx_smem<256, 16, T>());
      case 512: return go(k_fft_x_fwd_reg<512, 32, T, TV>, 16, fx_rows<512, 32>(), fx_smem<512, 32, T>());
      default: break;
    }
  }
  dim3 blk, grd;
  size_t smem;
  fft_x_shape<T>(g, blk, grd, smem);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_fft_x_fwd<T, TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_fft_x_fwd<T, TV><<<grd, blk, smem, s>>>(a, g, m, spec, tw_half, tw_post);
  return cudaGetLastError();
}

// Inverse x-transform (complex N/2+1 -> real N), times N (no normalisation).
template <typename T, typename TO>
__global__ void k_fft_x_inv(PoissonDst dst, const cplx<T>* __restrict__ spec, Geo g, Metrics m,
                            const cplx<T>* __restrict__ tw_half, const cplx<T>* __restrict__ tw_post,
                            double V, TO* __restrict__ out, const double* __restrict__ plane_add,
                            const TO* __restrict__ cell_add) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* sm = reinterpret_cast<cplx<T>*>(smem_raw);
  const int Lh = g.nx >> 1;
  const int nrows = g.nyc * g.nz;
  const int row = blockIdx.x * blockDim.y + threadIdx.y;
  cplx<T>* xa = sm + (size_t)threadIdx.y * 2 * Lh;
  cplx<T>* xb = xa + Lh;
  const bool live = row < nrows;
  const cplx<T>* in = spec + (size_t)(live ? row : 0) * g.mp;
  for (int mm = threadIdx.x; mm < Lh; mm += blockDim.x) {
    cplx<T> z = {T(0), T(0)};
    if (live) {
      const cplx<T> Xm = in[mm];
      const cplx<T> Xc = cconj(in[Lh - mm]);
      const cplx<T> sum = cadd(Xm, Xc);
      const cplx<T> dif = csub(Xm, Xc);
      const cplx<T> t = cmul(cconj(tw_post[mm]), dif);
      z = {sum.x - t.y, sum.y + t.x};   // sum + i * t
    }
    xa[mm] = z;
  }
  __syncthreads();
  cplx<T>* Z = stockham(xa, xb, Lh, tw_half, true, threadIdx.x, blockDim.x);
  if (!live) return;
  const int j = row / g.nz;
  const size_t base = (size_t)row * g.nx;
  const double add = dst == PoissonDst::Potential ? V * m.yc[j] : 0.0;
  const T addT = dst == PoissonDst::PotentialShadow ? (T)plane_add[j] : T(0);
  for (int t = threadIdx.x; t < Lh; t += blockDim.x) {
    const cplx<T> z = Z[t];
    if (dst == PoissonDst::PotentialShadow) {
      TO a0 = (TO)(addT + z.x), a1 = (TO)(addT + z.y);
      if (cell_add) { a0 += cell_add[base + 2 * t]; a1 += cell_add[base + 2 * t + 1]; }
      out[base + 2 * t] = a0;
      out[base + 2 * t + 1] = a1;
    } else if (dst == PoissonDst::Potential) {
      TO a0 = (TO)(add + (double)z.x), a1 = (TO)(add + (double)z.y);
      if (cell_add) { a0 += cell_add[base + 2 * t]; a1 += cell_add[base + 2 * t + 1]; }
      out[base + 2 * t] = a0;
      out[base + 2 * t + 1] = a1;
    } else {
      out[base + 2 * t] = (TO)z.x;
      out[base + 2 * t + 1] = (TO)z.y;
    }
  }
}

template <typename T, typename TO>
cudaError_t launch_fft_x_inv(PoissonDst dst, const cplx<T>* spec, const Geo& g, const Metrics& m,
                             const cplx<T>* tw_half, const cplx<T>* tw_post, double V, TO* out,
                             cudaStream_t s, const double* plane_add, const TO* cell_add) {
  {
    auto go = [&](auto kern, int G, int rows, size_t smem) {
      if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
      }
      const int nrows = g.nyc * g.nz;
      kern<<<(nrows + rows - 1) / rows, dim3(G, rows), smem, s>>>(dst, spec, g, m, tw_half, tw_post, V, out, plane_add,
                                                                  cell_add);
      return cudaGetLastError();
    };
    switch (g.nx / 2) {
      case 16: return go(k_fft_x_inv_reg<16, 4, T, TO>, 4, fx_rows<16, 4>(), fx_smem<16, 4, T>());
      case 32: return go(k_fft_x_inv_reg<32, 8, T, TO>, 4, fx_rows<32, 8>(), fx_smem<32, 8, T>());
      case 64: return go(k_fft_x_inv_reg<64, 8, T, TO>, 8, fx_rows<64, 8>(), fx_smem<64, 8, T>());
      case 128: return go(k_fft_x_inv_reg<128, 16, T, TO>, 8, fx_rows<128, 16>(), fx_smem<128, 16, T>());
      case 256: return go(k_fft_x_inv_reg<256, 16, T, TO>, 16, fx_rows<256, 16>(), fx_smem<256, 16, T>());
      case 512: return go(k_fft_x_inv_reg<512, 32, T, TO>, 16, fx_rows<512, 32>(), fx_smem<512, 32, T>());
      default: break;
    }
  }
  dim3 blk, grd;
  size_t smem;
  fft_x_shape<T>(g, blk, grd, smem);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_fft_x_inv<T, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_fft_x_inv<T, TO><<<grd, blk, smem, s>>>(dst, spec, g, m, tw_half, tw_post, V, out, plane_add, cell_add);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// z-transform of spectral columns: a block loads TM consecutive m-columns of
// one y-plane (TM complex values contiguous per z-row), transforms each
// column of length Nz in shared memory and writes it back in place.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_fft_z(cplx<T>* __restrict__ spec, const cplx<T>* __restrict__ tw_z, Geo g, bool inverse) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* sm = reinterpret_cast<cplx<T>*>(smem_raw);
  const int TM = blockDim.x;
  const int nz = g.nz;
  const int m0 = blockIdx.x * TM;
  const int j = blockIdx.y;
  const int tm = threadIdx.x;
  const int stride = nz + 1;   // padding against bank conflicts
  cplx<T>* xa = sm + (size_t)tm * stride;
  cplx<T>* xb = sm + (size_t)TM * stride + (size_t)tm * stride;
  const int m = m0 + tm;
  const bool live = m < g.mh;
  cplx<T>* plane = spec + (size_t)j * nz * g.mp;
  for (int n = threadIdx.y; n < nz; n += blockDim.y) {
    cplx<T> z = {T(0), T(0)};
    if (live) z = plane[(size_t)n * g.mp + m];
    xa[n] = z;
  }
  __syncthreads();
  cplx<T>* Z = stockham(xa, xb, nz, tw_z, inverse, threadIdx.y, blockDim.y);
  if (!live) return;
  for (int n = threadIdx.y; n < nz; n += blockDim.y) plane[(size_t)n * g.mp + m] = Z[n];
}

// z-transform with the two-pass register FFT (pnp_regfft.cuh), FP32 or FP64: a block
// owns TM consecutive m-columns of one y-plane; thread (tm, g) loads the
// samples n = g + G r of column tm (TM-wide coalesced rows), does the R1-point
// DFT in registers, multiplies by W_N^{g k1} and exchanges through shared
// memory; thread g then does the G-point DFTs of its R1 / G values of k1 and
// stores X[k1 + R1 k2].
template <int N, int R1, int TM, bool INV, typename T>
__global__ void __launch_bounds__(TM*(N / R1)) k_fft_z_reg(cplx<T>* __restrict__ spec,
                                                           const cplx<T>* __restrict__ tw, Geo g) {
  constexpr int G = N / R1, PER = R1 / G;
  static_assert(R1 % G == 0, "each thread takes whole G-point transforms");
  extern __shared__ __align__(16) unsigned char fz_smem[];
  cplx<T>* xs = reinterpret_cast<cplx<T>*>(fz_smem);   // [TM][N + 1] (padded against bank conflicts)
  cplx<T>* twl = xs + TM * (N + 1);                      // [N]
  const int tm = threadIdx.x, gi = threadIdx.y, tid = gi * TM + tm;
  for (int e = tid; e < N; e += TM * G) {
    cplx<T> t = tw[e];
    if (INV) t.y = -t.y;
    twl[e] = t;
  }
  const int m = blockIdx.x * TM + tm;
  const bool live = m < g.mh;
  cplx<T>* col = spec + (size_t)blockIdx.y * N * g.mp + (live ? m : 0);
  cplx<T> v[R1];
#pragma unroll
  for (int r = 0; r < R1; ++r) v[r] = live ? col[(size_t)(gi + G * r) * g.mp] : cplx<T>{T(0), T(0)};
  __syncthreads();   // the twiddle table
  rfft::dft<INV, R1>(v);
  cplx<T>* xm = xs + tm * (N + 1);
  rfft::static_for<0, R1>([&](auto kc) {
    constexpr int k1 = decltype(kc)::value;
    xm[k1 * G + gi] = cmul(v[rfft::bitrev(k1, R1)], twl[gi * k1]);
  });
  __syncthreads();
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int k1 = gi * PER + p;
    cplx<T> w[G];
#pragma unroll
    for (int q = 0; q < G; ++q) w[q] = xm[k1 * G + q];
    rfft::dft<INV, G>(w);
    if (live) {
      rfft::static_for<0, G>([&](auto kc) {
        constexpr int k2 = decltype(kc)::value;
        col[(size_t)(k1 + R1 * k2) * g.mp] = w[rfft::bitrev(k2, G)];
      });
    }
  }
}

template <int N, int R1, int TM, typename T>
cudaError_t launch_fft_z_reg(cplx<T>* spec, const cplx<T>* tw, const Geo& g, bool inverse, cudaStream_t s) {
  constexpr int G = N / R1;
  const size_t smem = sizeof(cplx<T>) * ((size_t)TM * (N + 1) + N);
  const dim3 grd((unsigned)((g.mh + TM - 1) / TM), (unsigned)g.nyc);
  auto go = [&](auto kern) {
    if (smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    kern<<<grd, dim3(TM, G), smem, s>>>(spec, tw, g);
    return cudaGetLastError();
  };
  return inverse ? go(k_fft_z_reg<N, R1, TM, true, T>) : go(k_fft_z_reg<N, R1, TM, false, T>);
}

template <typename T>
cudaError_t launch_fft_z(cplx<T>* spec, const cplx<T>* tw_z, const Geo& g, bool inverse, cudaStream_t s) {
  // register transforms for 16 <= Nz <= 512 unless the stage-by-stage kernel is asked for
  if (g.lc_fftz_ty != 64) {
    switch (g.nz) {
      case 16: return launch_fft_z_reg<16, 4, 32, T>(spec, tw_z, g, inverse, s);
      case 32: return launch_fft_z_reg<32, 8, 32, T>(spec, tw_z, g, inverse, s);
      case 64: return launch_fft_z_reg<64, 8, 32, T>(spec, tw_z, g, inverse, s);
      case 128: return launch_fft_z_reg<128, 16, 32, T>(spec, tw_z, g, inverse, s);
      case 256: return launch_fft_z_reg<256, 16, 16, T>(spec, tw_z, g, inverse, s);
      case 512: return launch_fft_z_reg<512, 32, 8, T>(spec, tw_z, g, inverse, s);
      default: break;
    }
  }
  int TM = (int)(128 / sizeof(cplx<T>));   // one 128-byte segment of each z-row
  while (TM > 1 && (size_t)2 * TM * (g.nz + 1) * sizeof(cplx<T>) > 200 * 1024) TM >>= 1;
  int ty = g.nz / 4;
  const int cap = g.lc_fftz_ty ? g.lc_fftz_ty : 32;
  if (ty > cap) ty = cap;
  if (ty < 1) ty = 1;
  dim3 blk(TM, ty, 1);
  dim3 grd((g.mh + TM - 1) / TM, g.nyc, 1);
  const size_t smem = (size_t)2 * TM * (g.nz + 1) * sizeof(cplx<T>);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_fft_z<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_fft_z<T><<<grd, blk, smem, s>>>(spec, tw_z, g, inverse);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Spectral Thomas: per (m, n), solve a_j x_{j-1} + (b_j - kx2_m - kz2_n) x_j
// + c_j x_{j+1} = scale * rhs_j in FP64.  The Neumann (0,0) mode replaces its
// bottom-row equation by x_0 = 0.  The elimination factors depend only on the
// grid, so they are computed once (k_spec_factors): inv_j = 1 / (B_j - a_j
// c'_{j-1}) and c'_j = c_j inv_j, stored per spectral point in FP64.
// The sweeps load CH planes ahead so that a thread keeps CH independent
// memory requests in flight instead of one per serial step.
// ---------------------------------------------------------------------------
__global__ void k_spec_factors(double* __restrict__ cpr, double* __restrict__ inv, const double* __restrict__ kx2,
                               const double* __restrict__ kz2, YRows rows, Geo g, bool neumann) {
  const int mm = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = blockIdx.y;
  if (mm >= g.mh) return;
  const size_t P = (size_t)g.nz * g.mp;
  const size_t base = (size_t)n * g.mp + mm;
  const double k2 = kx2[mm] + kz2[n];
  const bool pin = neumann && mm == 0 && n == 0;
  double cprev = 0.0;
  for (int j = 0; j < g.nyc; ++j) {
    double a = rows.a[j], b = rows.b[j] - k2, c = rows.c[j];
    if (pin && j == 0) { b = 1.0; c = 0.0; }
    const double iv = 1.0 / (b - a * cprev);
    cprev = c * iv;
    cpr[base + (size_t)j * P] = cprev;
    inv[base + (size_t)j * P] = iv;
  }
}

cudaError_t launch_spec_factors(double* cpr, double* inv, const double* kx2, const double* kz2, const YRows& rows,
                                const Geo& g, bool neumann, cudaStream_t s) {
  const int T_ = 64;
  dim3 grd((g.mh + T_ - 1) / T_, g.nz, 1);
  k_spec_factors<<<grd, T_, 0, s>>>(cpr, inv, kx2, kz2, rows, g, neumann);
  return cudaGetLastError();
}

constexpr int kCH = 8;

// FP64 (0,0) mode of the mixed potential: the FP32 transform's mean of the
// fluctuating charge, scaled, plus the FP64 reference source; the solution goes
// to mean_out (plus mean_shift) and the transform slot is zeroed.  Runs in the
// real-part thread; the imaginary-part thread only zeroes its slots.
template <typename T>
__device__ void spec_mean_mode(T* sp, const double* __restrict__ cpr, const double* __restrict__ inv,
                               const YRows& rows, size_t base, size_t P, int ny, int part, double scale,
                               const double* __restrict__ mean_rhs, const double* __restrict__ mean_shift,
                               double* __restrict__ mean_out) {
  if (part == 1) {
    for (int j = 0; j < ny; ++j) sp[2 * (base + (size_t)j * P)] = T(0);
    return;
  }
  double d = 0.0;
  for (int j0 = 0; j0 < ny; j0 += kCH) {
    double rr[kCH], iv[kCH], mr[kCH];
#pragma unroll
    for (int u = 0; u < kCH; ++u)
      if (j0 + u < ny) {
        const size_t o = base + (size_t)(j0 + u) * P;
        rr[u] = (double)sp[2 * o];
        iv[u] = inv[o];
        mr[u] = mean_rhs[j0 + u];
      }
#pragma unroll
    for (int u = 0; u < kCH; ++u)
      if (j0 + u < ny) {
        d = (rr[u] * scale + mr[u] - rows.a[j0 + u] * d) * iv[u];
        mean_out[j0 + u] = d;
      }
  }
  double x = d;
  mean_out[ny - 1] = x + mean_shift[ny - 1];
  sp[2 * (base + (size_t)(ny - 1) * P)] = T(0);
  for (int j1 = ny - 2; j1 >= 0; j1 -= kCH) {
    double dd[kCH], cc[kCH], ms[kCH];
#pragma unroll
    for (int u = 0; u < kCH; ++u)
      if (j1 - u >= 0) {
        dd[u] = mean_out[j1 - u];
        cc[u] = cpr[base + (size_t)(j1 - u) * P];
        ms[u] = mean_shift[j1 - u];
      }
#pragma unroll
    for (int u = 0; u < kCH; ++u)
      if (j1 - u >= 0) {
        x = dd[u] - cc[u] * x;
        mean_out[j1 - u] = x + ms[u];
        sp[2 * (base + (size_t)(j1 - u) * P)] = T(0);
      }
  }
}

// The forward sweep runs on the unscaled transform; its FP64 results go to an
// FP64 scratch (no round trip through the transform's precision), and the
// normalisation 1/(Nx Nz) is applied once, in the transform's precision, when
// the solution is stored.  The real and imaginary parts are independent
// recurrences with the same coefficients, so each runs in its own thread
// (adjacent threads touch the two halves of one complex value).  The FP64 mean
// mode (mixed potential) keeps the scaled physical source and never touches
// spec; it runs in the real-part thread of (0,0).
template <typename T>
__global__ void k_spec_thomas(cplx<T>* __restrict__ spec, cplx<double>* __restrict__ dscr,
                              const double* __restrict__ cpr, const double* __restrict__ inv, YRows rows, Geo g,
                              double scale, bool neumann, const double* __restrict__ mean_rhs,
                              const double* __restrict__ mean_shift, double* __restrict__ mean_out) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int mm = tid >> 1, part = tid & 1;
  const int n = blockIdx.y;
  if (mm >= g.mh) return;
  const size_t P = (size_t)g.nz * g.mp;
  const size_t base = (size_t)n * g.mp + mm;
  const int ny = g.nyc;
  T* sp = reinterpret_cast<T*>(spec) + part;             // this part of spec[base + j P] at sp[2 (base + j P)]
  double* dp = reinterpret_cast<double*>(dscr) + part;
  const bool pin = neumann && mm == 0 && n == 0;
  const bool mean_mode = mean_rhs != nullptr && mm == 0 && n == 0;
  if (mean_mode) {
    spec_mean_mode(sp, cpr, inv, rows, base, P, ny, part, scale, mean_rhs, mean_shift, mean_out);
    return;
  }
  double d = 0.0;
  for (int j0 = 0; j0 < ny; j0 += kCH) {
    double rr[kCH], iv[kCH];
#pragma unroll
    for (int u = 0; u < kCH; ++u) {
      if (j0 + u < ny) {
        const size_t o = base + (size_t)(j0 + u) * P;
        rr[u] = (double)sp[2 * o];
        iv[u] = inv[o];
      }
    }
#pragma unroll
    for (int u = 0; u < kCH; ++u) {
      const int j = j0 + u;
      if (j < ny) {
        const double r = (pin && j == 0) ? 0.0 : rr[u];
        d = (r - rows.a[j] * d) * iv[u];
        dp[2 * (base + (size_t)j * P)] = d;
      }
    }
  }
  const T sc = (T)scale;
  double x = d;
  sp[2 * (base + (size_t)(ny - 1) * P)] = (T)x * sc;
  for (int j1 = ny - 2; j1 >= 0; j1 -= kCH) {
    double dd[kCH], cc[kCH];
#pragma unroll
    for (int u = 0; u < kCH; ++u) {
      if (j1 - u >= 0) {
        const size_t o = base + (size_t)(j1 - u) * P;
        dd[u] = dp[2 * o];
        cc[u] = cpr[o];
      }
    }
#pragma unroll
    for (int u = 0; u < kCH; ++u) {
      const int j = j1 - u;
      if (j >= 0) {
        x = dd[u] - cc[u] * x;
        sp[2 * (base + (size_t)j * P)] = (T)x * sc;
      }
    }
  }
}

template <typename T>
cudaError_t launch_spec_thomas(cplx<T>* spec, cplx<double>* dscr, const double* cpr, const double* inv,
                               const YRows& rows, const Geo& g, double scale, bool neumann, cudaStream_t s,
                               const double* mean_rhs, const double* mean_shift, double* mean_out) {
  const int T_ = g.lc_spec ? g.lc_spec : 64;
  dim3 grd((2 * g.mh + T_ - 1) / T_, g.nz, 1);
  k_spec_thomas<T><<<grd, T_, 0, s>>>(spec, dscr, cpr, inv, rows, g, scale, neumann, mean_rhs, mean_shift, mean_out);
  return cudaGetLastError();
}

// Rows per batch of the df line sweeps (two batches in flight per thread).
constexpr int kDfCH = 4;

// Mixed path: the same elimination in double-float arithmetic on the FP32 pipe
// (pnp_df.cuh).  The low wavenumbers are ill-conditioned on the stretched grid
// (the near-wall rows dominate |A| |x| by orders of magnitude over A x), so the
// recurrence needs more than FP32; df carries a 48-bit significand at a small
// fraction of the FP64 pipe time.  Factors c'_j, 1/pivot_j and the
// sub-diagonal a_j arrive as df pairs (converted once from the FP64 factors);
// the forward-sweep values go to the scratch as df pairs; the (0,0) mode of the
// mixed potential keeps its FP64 path.
__global__ void k_spec_thomas_df(cplx<float>* __restrict__ spec, float2* __restrict__ dscr,
                                 const float2* __restrict__ cprF, const float2* __restrict__ invF,
                                 const float2* __restrict__ aF, const double* __restrict__ cpr,
                                 const double* __restrict__ inv, YRows rows, Geo g, double scale, float sc,
                                 bool neumann, const double* __restrict__ mean_rhs,
                                 const double* __restrict__ mean_shift, double* __restrict__ mean_out) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int mm = tid >> 1, part = tid & 1;
  const int n = blockIdx.y;
  if (mm >= g.mh) return;
  const size_t P = (size_t)g.nz * g.mp;
  const size_t base = (size_t)n * g.mp + mm;
  const int ny = g.nyc;
  float* sp = reinterpret_cast<float*>(spec) + part;   // this part of spec[base + j P] at sp[2 (base + j P)]
  float2* dp = dscr + part;                             // its df forward value at dp[2 (base + j P)]
  const bool pin = neumann && mm == 0 && n == 0;
  if (mean_rhs != nullptr && mm == 0 && n == 0) return;   // k_spec_mean handles the (0,0) mode
  // Both sweeps run in kDfCH-row batches, double-buffered: the loads of batch
  // b + 1 are in flight while batch b's recurrence runs.
  auto load_f = [&](int j0, float (&rr)[kDfCH], float2 (&iv)[kDfCH]) {
#pragma unroll
    for (int u = 0; u < kDfCH; ++u)
      if (j0 + u < ny) {
        const size_t o = base + (size_t)(j0 + u) * P;
        rr[u] = sp[2 * o];
        iv[u] = invF[o];
      }
  };
  auto comp_f = [&](int j0, const float (&rr)[kDfCH], const float2 (&iv)[kDfCH], dfl d) {
#pragma unroll
    for (int u = 0; u < kDfCH; ++u) {
      const int j = j0 + u;
      if (j < ny) {
        const float r = (pin && j == 0) ? 0.f : rr[u];
        const float2 a = aF[j];
        d = df_mul(df_sub_mul(r, dfl{a.x, a.y}, d), dfl{iv[u].x, iv[u].y});
        if (j < ny - 1) dp[2 * (base + (size_t)j * P)] = make_float2(d.h, d.l);
      }
    }
    return d;
  };
  dfl d{0.f, 0.f};
  {
    float rA[kDfCH], rB[kDfCH];
    float2 iA[kDfCH], iB[kDfCH];
    load_f(0, rA, iA);
    for (int j0 = 0; j0 < ny; j0 += 2 * kDfCH) {
      if (j0 + kDfCH < ny) load_f(j0 + kDfCH, rB, iB);
      d = comp_f(j0, rA, iA, d);
      if (j0 + kDfCH < ny) {
        if (j0 + 2 * kDfCH < ny) load_f(j0 + 2 * kDfCH, rA, iA);
        d = comp_f(j0 + kDfCH, rB, iB, d);
      }
    }
  }
  dfl x = d;
  sp[2 * (base + (size_t)(ny - 1) * P)] = x.h * sc;
  // back substitution over rows j1, j1 - 1, ..., j1 - kDfCH + 1 (those >= 0)
  auto load_b = [&](int j1, float2 (&dd)[kDfCH], float2 (&cc)[kDfCH]) {
#pragma unroll
    for (int u = 0; u < kDfCH; ++u)
      if (j1 - u >= 0) {
        const size_t o = base + (size_t)(j1 - u) * P;
        dd[u] = dp[2 * o];
        cc[u] = cprF[o];
      }
  };
  auto comp_b = [&](int j1, const float2 (&dd)[kDfCH], const float2 (&cc)[kDfCH], dfl x) {
#pragma unroll
    for (int u = 0; u < kDfCH; ++u) {
      const int j = j1 - u;
      if (j >= 0) {
        x = df_sub_mul(dfl{dd[u].x, dd[u].y}, dfl{cc[u].x, cc[u].y}, x);
        sp[2 * (base + (size_t)j * P)] = x.h * sc;
      }
    }
    return x;
  };
  {
    float2 dA[kDfCH], dB[kDfCH], cA[kDfCH], cB[kDfCH];
    load_b(ny - 2, dA, cA);
    for (int j1 = ny - 2; j1 >= 0; j1 -= 2 * kDfCH) {
      if (j1 - kDfCH >= 0) load_b(j1 - kDfCH, dB, cB);
      x = comp_b(j1, dA, cA, x);
      if (j1 - kDfCH >= 0) {
        if (j1 - 2 * kDfCH >= 0) load_b(j1 - 2 * kDfCH, dA, cA);
        x = comp_b(j1 - kDfCH, dB, cB, x);
      }
    }
  }
}

// The FP64 (0,0) mode of the mixed potential as one block.  All threads stage
// the column in shared memory; both Thomas sweeps are first-order linear
// recurrences x_j = A_j + B_j x_(j-1) (forward: A = src_j / pivot_j,
// B = -a_j / pivot_j; back substitution, run from the top: A = d_j, B = -c'_j),
// so the first warp solves each as a scan of affine maps: every lane composes
// the maps of its chunk of rows, a Kogge-Stone scan over the 32 lanes composes
// the chunks, and every lane re-runs its chunk from the value entering it.
// The dependent FP64 chain shrinks from two steps per row to ~2 n / 32 + 10
// steps.  |B| < 1 on the diagonally dominant y-operator, so the composed
// products only shrink.  Then all threads write the result and zero the
// transform slots.
constexpr int kMeanSmemRows = 640;   // 5 doubles per row: 25 KB of static shared memory

// x_j = A_j + B_j x_(j-1) for j = 0 .. n-1 with x_(-1) = 0, by the first warp;
// A(s), B(s) give the maps in sweep order s, x(s, value) stores the result
template <typename FA, typename FB, typename FX>
__device__ __forceinline__ void affine_scan_warp(int n, FA A, FB B, FX x) {
  const int lane = threadIdx.x & 31, per = (n + 31) / 32;
  const int lo = min(n, lane * per), hi = min(n, lo + per);
  double bc = 1.0, ac = 0.0;   // this chunk's composed map
  for (int s = lo; s < hi; ++s) {
    const double b = B(s);
    ac = fma(b, ac, A(s));
    bc *= b;
  }
  // inclusive scan over lanes: (b, a) of lanes <= lane composed, earlier first
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const double bp = __shfl_up_sync(0xffffffffu, bc, off), ap = __shfl_up_sync(0xffffffffu, ac, off);
    if (lane >= off) {
      ac = fma(bc, ap, ac);
      bc *= bp;
    }
  }
  double v = __shfl_up_sync(0xffffffffu, ac, 1);   // the value entering this chunk
  if (lane == 0) v = 0.0;
  for (int s = lo; s < hi; ++s) {
    v = fma(B(s), v, A(s));
    x(s, v);
  }
}

__global__ void __launch_bounds__(256) k_spec_mean(cplx<float>* __restrict__ spec, const double* __restrict__ cpr,
                                                   const double* __restrict__ inv, YRows rows, Geo g, double scale,
                                                   const double* __restrict__ mean_rhs,
                                                   const double* __restrict__ mean_shift,
                                                   double* __restrict__ mean_out) {
  const size_t P = (size_t)g.nz * g.mp;
  const int ny = g.nyc;
  float* sp = reinterpret_cast<float*>(spec);   // (0,0) mode, real part at sp[2 j P], imaginary at sp[2 j P + 1]
  if (ny > kMeanSmemRows) {
    if (threadIdx.x < 2)
      spec_mean_mode(sp + threadIdx.x, cpr, inv, rows, 0, P, ny, (int)threadIdx.x, scale, mean_rhs, mean_shift,
                     mean_out);
    return;
  }
  __shared__ double e[kMeanSmemRows], fa[kMeanSmemRows], cp[kMeanSmemRows], ms[kMeanSmemRows],
      out[kMeanSmemRows];
  for (int j = threadIdx.x; j < ny; j += blockDim.x) {
    const size_t o = (size_t)j * P;
    const double iv = inv[o];
    e[j] = ((double)sp[2 * o] * scale + mean_rhs[j]) * iv;
    fa[j] = rows.a[j] * iv;
    cp[j] = cpr[o];
    ms[j] = mean_shift[j];
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // forward: d_j = e_j - (a_j / pivot_j) d_(j-1)
    affine_scan_warp(ny, [&](int s) { return e[s]; }, [&](int s) { return -fa[s]; },
                     [&](int s, double v) { out[s] = v; });
    __syncwarp();
    // back substitution from the top: x_(n-1) = d_(n-1), x_j = d_j - c'_j x_(j+1)
    affine_scan_warp(ny, [&](int s) { return out[ny - 1 - s]; },
                     [&](int s) { return s == 0 ? 0.0 : -cp[ny - 1 - s]; },
                     [&](int s, double v) { out[ny - 1 - s] = v; });
  }
  __syncthreads();
  for (int j = threadIdx.x; j < ny; j += blockDim.x) {
    const size_t o = (size_t)j * P;
    mean_out[j] = out[j] + ms[j];
    sp[2 * o] = 0.f;
    sp[2 * o + 1] = 0.f;
  }
}

// The same df elimination with the forward values in shared memory.  One warp
// owns 8 consecutive spectral points m of two z-wavenumbers n (16 points, real
// and imaginary part in adjacent lanes); the right-hand sides and 1/pivot of
// the forward sweep, then c' of the back substitution, stream through a
// two-chunk cp.async ring (16 planes per chunk, the back-substitution chunks
// following the forward ones without a gap), and the df values d_j stay in
// shared memory, so the sweep scratch never reaches HBM.  Same operations in
// the same order as k_spec_thomas_df.
constexpr int kSpChunk = 16;

__host__ __device__ inline size_t spec_tile_bytes(int n) {
  // d [n][32] float2, r ring [2][kSpChunk][32] float, factor ring [2][kSpChunk][16] float2, a [n] float2
  return (size_t)n * 32 * 8 + 2 * kSpChunk * 32 * 4 + 2 * kSpChunk * 16 * 8 + (size_t)n * 8;
}

__device__ __forceinline__ void sp_cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

__global__ void __launch_bounds__(32) k_spec_thomas_tile(cplx<float>* __restrict__ spec, SpecDF f, Geo g, float sc,
                                                         bool neumann, bool skip_mean) {
  extern __shared__ __align__(16) unsigned char sp_smem[];
  const int n = g.nyc;
  float2* dd = reinterpret_cast<float2*>(sp_smem);              // [n][32]
  float* rr = reinterpret_cast<float*>(dd + (size_t)n * 32);    // [2][kSpChunk][32]
  float2* ff = reinterpret_cast<float2*>(rr + 2 * kSpChunk * 32);   // [2][kSpChunk][16]
  float2* aa = ff + 2 * kSpChunk * 16;                          // [n]
  const int t = threadIdx.x, part = t & 1, q = t >> 1, rs = q >> 3, mq = q & 7;
  const int m0 = blockIdx.x * 8, n0 = blockIdx.y * 2;
  const int m = m0 + mq, nn = n0 + rs;
  const size_t P = (size_t)g.nz * g.mp;   // complex values per plane
  const float* specf = reinterpret_cast<const float*>(spec);
  const int K = (n + kSpChunk - 1) / kSpChunk;
  // step s < K: forward chunk s (r and 1/pivot of planes [16 s, 16 s + 16));
  // step s >= K: back-substitution chunk b = s - K (c' of planes [hi - 16, hi), hi = n - 16 b)
  auto issue = [&](int st) {
    if (st < 2 * K) {
      const bool fwd = st < K;
      const int b = fwd ? st : st - K;
      const int hi = fwd ? min(n, (b + 1) * kSpChunk) : n - b * kSpChunk;
      const int lo = fwd ? b * kSpChunk : max(0, hi - kSpChunk);
      float* rb = rr + (st & 1) * kSpChunk * 32;
      float2* fb = ff + (st & 1) * kSpChunk * 16;
      const float2* fac = fwd ? f.inv : f.cpr;
      for (int e = t; e < (hi - lo) * 8; e += 32) {
        const int jj = e >> 3, sr = (e >> 2) & 1, c = e & 3;
        const int j = fwd ? lo + jj : hi - 1 - jj;
        const size_t o = (size_t)j * P + (size_t)(n0 + sr) * g.mp + m0;   // complex index of the row segment
        if (fwd) sp_cp_async16(rb + jj * 32 + sr * 16 + c * 4, specf + 2 * o + c * 4);
        sp_cp_async16(fb + jj * 16 + sr * 8 + c * 2, fac + o + c * 2);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  issue(0);
  issue(1);
  for (int j = t; j < n; j += 32) aa[j] = f.a[j];
  const bool pin = neumann && m == 0 && nn == 0;
  dfl d{0.f, 0.f};
  for (int st = 0; st < K; ++st) {
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncwarp();
    const float* rb = rr + (st & 1) * kSpChunk * 32;
    const float2* fb = ff + (st & 1) * kSpChunk * 16;
    const int lo = st * kSpChunk, hi = min(n, lo + kSpChunk);
    for (int j = lo; j < hi; ++j) {
      const int jj = j - lo;
      const float r = (pin && j == 0) ? 0.f : rb[jj * 32 + t];
      const float2 a = aa[j], iv = fb[jj * 16 + q];
      d = df_mul(df_sub_mul(r, dfl{a.x, a.y}, d), dfl{iv.x, iv.y});
      dd[(size_t)j * 32 + t] = make_float2(d.h, d.l);
    }
    __syncwarp();
    issue(st + 2);
  }
  const bool store = m < g.mh && !(skip_mean && m == 0 && nn == 0);
  float* out = reinterpret_cast<float*>(spec) + 2 * ((size_t)nn * g.mp + m) + part;   // plane j at out[2 j P]
  dfl x = d;
  for (int b = 0; b < K; ++b) {
    const int st = K + b;
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncwarp();
    const float2* fb = ff + (st & 1) * kSpChunk * 16;
    const int hi = n - b * kSpChunk, lo = max(0, hi - kSpChunk);
    for (int j = hi - 1; j >= lo; --j) {
      if (j < n - 1) {
        const float2 dj = dd[(size_t)j * 32 + t], cp = fb[(hi - 1 - j) * 16 + q];
        x = df_sub_mul(dfl{dj.x, dj.y}, dfl{cp.x, cp.y}, x);
      }
      if (store) out[2 * (size_t)j * P] = x.h * sc;
    }
    __syncwarp();
    issue(st + 2);
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

cudaError_t launch_spec_thomas_df(cplx<float>* spec, void* dscr, const SpecDF& f, const double* cpr,
                                  const double* inv, const YRows& rows, const Geo& g, double scale, bool neumann,
                                  cudaStream_t s, const double* mean_rhs, const double* mean_shift,
                                  double* mean_out) {
  if (mean_rhs != nullptr) {
    k_spec_mean<<<1, 256, 0, s>>>(spec, cpr, inv, rows, g, scale, mean_rhs, mean_shift, mean_out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // shared-memory tiles (lc_spec 16) when 8-point row segments tile the padded
  // pitch, the z-wavenumbers pair up and a column block fits.  Measured on the
  // 256x193x256 workload: 0.18 ms against 0.10 ms for one thread per point --
  // the ~48 KB of df forward values per warp leaves three warps per SM to hide
  // the double-float dependency chain -- so it is only an autotuner candidate.
  const size_t tbytes = spec_tile_bytes(g.nyc);
  if (g.lc_spec == 16 && g.mp % 8 == 0 && g.nz % 2 == 0 && tbytes <= 227 * 1024) {
    if (tbytes > 48 * 1024) {
      const cudaError_t e =
          cudaFuncSetAttribute(k_spec_thomas_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tbytes);
      if (e != cudaSuccess) return e;
    }
    const dim3 grd((unsigned)((g.mh + 7) / 8), (unsigned)(g.nz / 2));
    k_spec_thomas_tile<<<grd, 32, tbytes, s>>>(spec, f, g, (float)scale, neumann, mean_rhs != nullptr);
    return cudaGetLastError();
  }
  const int T_ = g.lc_spec ? g.lc_spec : 64;
  dim3 grd((2 * g.mh + T_ - 1) / T_, g.nz, 1);
  k_spec_thomas_df<<<grd, T_, 0, s>>>(spec, reinterpret_cast<float2*>(dscr), f.cpr, f.inv, f.a, cpr, inv, rows, g,
                                      scale, (float)scale, neumann, mean_rhs, mean_shift, mean_out);
  return cudaGetLastError();
}

// x -> (hi, lo) float pairs, hi the nearest float.
__global__ void k_to_df(const double* __restrict__ x, float2* __restrict__ out, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  const float h = (float)v;
  out[i] = make_float2(h, (float)(v - (double)h));
}

cudaError_t launch_to_df(const double* x, float2* out, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_to_df<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, out, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Projection: u -= scale d(phip)/dx, w -= scale d(phip)/dz, v -= scale
// d(phip)/dy on interior faces; optionally p += phip.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_project(T* __restrict__ u, T* __restrict__ v, T* __restrict__ w, T* __restrict__ p,
                          const T* __restrict__ s, T cx, T cz, T sc, const T* __restrict__ ih, bool update_p, Geo g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.z;
  if (i >= g.nx || k >= g.nz) return;
  const int im = i ? i - 1 : g.nx - 1;
  const int km = k ? k - 1 : g.nz - 1;
  const size_t c = cidx(j, k, i, g.nz, g.nx);
  const T s0 = s[c];
  u[c] = u[c] - cx * (s0 - s[cidx(j, k, im, g.nz, g.nx)]);
  w[c] = w[c] - cz * (s0 - s[cidx(j, km, i, g.nz, g.nx)]);
  if (j > 0) v[c] = v[c] - sc * (s0 - s[c - (size_t)g.nz * g.nx]) * ih[j];
  if (update_p) p[c] = p[c] + s0;
}

// FP32 projection for x-rows of 128 cells: a warp owns 128 consecutive x-cells
// (a float4 per lane) of one z-row and marches a chunk of y-planes, carrying
// Phi_p of the plane below in registers; the x-neighbour of a lane's first cell
// is the previous lane's last (a shuffle; lane 0 wraps or loads it).
__global__ void __launch_bounds__(128) k_project_rows(float* __restrict__ u, float* __restrict__ v,
                                                     float* __restrict__ w, float* __restrict__ p,
                                                     const float* __restrict__ s, float cx, float cz, float sc,
                                                     const float* __restrict__ ih, bool update_p, Geo g, int jchunk) {
  const int lane = threadIdx.x, nx = g.nx, nz = g.nz;
  const int i0 = blockIdx.x * 128 + lane * 4;
  const int k = blockIdx.y * blockDim.y + threadIdx.y;
  const int jb = blockIdx.z * jchunk, je = min(g.nyc, jb + jchunk);
  const int km = k ? k - 1 : nz - 1;
  const size_t P = (size_t)nz * nx;
  const size_t row = (size_t)k * nx + i0, rowm = (size_t)km * nx + i0;
  // wrapped x-neighbour of the warp's first cell
  const size_t xwrap = (size_t)k * nx + (blockIdx.x == 0 ? nx - 1 : blockIdx.x * 128 - 1);
  float4 sb = make_float4(0.f, 0.f, 0.f, 0.f);   // Phi_p of plane j - 1
  if (jb > 0) sb = *reinterpret_cast<const float4*>(s + (size_t)(jb - 1) * P + row);
  // every operand of plane j; the loads of plane j + 1 are issued before plane
  // j's arithmetic, so each thread keeps two planes of loads in flight
  struct Plane {
    float4 s0, sz, uu, ww, vv, pp;
    float sxw;
  };
  auto load = [&](int j, Plane& q) {
    const size_t o = (size_t)j * P;
    q.s0 = *reinterpret_cast<const float4*>(s + o + row);
    q.sz = *reinterpret_cast<const float4*>(s + o + rowm);
    q.sxw = lane == 0 ? s[o + xwrap] : 0.f;
    q.uu = *reinterpret_cast<const float4*>(u + o + row);
    q.ww = *reinterpret_cast<const float4*>(w + o + row);
    if (j > 0) q.vv = *reinterpret_cast<const float4*>(v + o + row);
    if (update_p) q.pp = *reinterpret_cast<const float4*>(p + o + row);
  };
  Plane cur, nxt;
  if (jb < je) load(jb, cur);
  for (int j = jb; j < je; ++j) {
    if (j + 1 < je) load(j + 1, nxt);
    const size_t o = (size_t)j * P;
    const float4 s0 = cur.s0, sz = cur.sz;
    float sx = __shfl_up_sync(0xffffffffu, s0.w, 1);
    if (lane == 0) sx = cur.sxw;
    float4 uu = cur.uu, ww = cur.ww;
    uu.x -= cx * (s0.x - sx);
    uu.y -= cx * (s0.y - s0.x);
    uu.z -= cx * (s0.z - s0.y);
    uu.w -= cx * (s0.w - s0.z);
    ww.x -= cz * (s0.x - sz.x);
    ww.y -= cz * (s0.y - sz.y);
    ww.z -= cz * (s0.z - sz.z);
    ww.w -= cz * (s0.w - sz.w);
    *reinterpret_cast<float4*>(u + o + row) = uu;
    *reinterpret_cast<float4*>(w + o + row) = ww;
    if (j > 0) {
      const float hj = ih[j];
      float4 vv = cur.vv;
      vv.x -= sc * (s0.x - sb.x) * hj;
      vv.y -= sc * (s0.y - sb.y) * hj;
      vv.z -= sc * (s0.z - sb.z) * hj;
      vv.w -= sc * (s0.w - sb.w) * hj;
      *reinterpret_cast<float4*>(v + o + row) = vv;
    }
    if (update_p) {
      float4 pp = cur.pp;
      pp.x += s0.x;
      pp.y += s0.y;
      pp.z += s0.z;
      pp.w += s0.w;
      *reinterpret_cast<float4*>(p + o + row) = pp;
    }
    sb = s0;
    cur = nxt;
  }
}

template <typename T>
cudaError_t launch_project(T* u, T* v, T* w, T* p, const T* phip, double scale, bool update_p, const Geo& g,
                           const T* ih, cudaStream_t s) {
  if constexpr (sizeof(T) == sizeof(float)) {
    if (g.nx % 128 == 0 && g.nz % 4 == 0) {
      // y-chunks of about 2 planes: many short blocks, which share the GPU best
      // with the other stream's kernels (swept over 2-48 planes on the
      // 256x193x256 workload: 2 best, 2.592 against 2.595 ms per step at 4 and
      // 2.605 at 16)
      const int nch = (g.nyc + 1) / 2, jc = (g.nyc + nch - 1) / nch;
      const dim3 grd((unsigned)(g.nx / 128), (unsigned)(g.nz / 4), (unsigned)((g.nyc + jc - 1) / jc));
      k_project_rows<<<grd, dim3(32, 4), 0, s>>>(u, v, w, p, phip, (float)(scale * g.idx), (float)(scale * g.idz),
                                                 (float)scale, ih, update_p, g, jc);
      return cudaGetLastError();
    }
  }
  dim3 blk(32, 4, 1);
  dim3 grd((g.nx + 31) / 32, (g.nz + 3) / 4, g.nyc);
  k_project<T><<<grd, blk, 0, s>>>(u, v, w, p, phip, (T)(scale * g.idx), (T)(scale * g.idz), (T)scale, ih, update_p, g);
  return cudaGetLastError();
}

// ---- explicit instantiations ----
// ---------------------------------------------------------------------------
// Periodic x / z sweeps of the approximate factorisation.  A block stages L
// whole lines of one family in shared memory with coalesced loads (x: L rows
// of nx contiguous values; z: L adjacent columns of one plane, nz values each,
// read as L-wide row segments), thread t < L solves line t there (forward
// elimination, back substitution, Sherman-Morrison correction: the cyclic
// system's three passes never touch HBM), and the block writes the lines back.
// ---------------------------------------------------------------------------
template <typename T, bool ZDIR>
__global__ void __launch_bounds__(128) k_periodic(PeriodicArgs<T> A, Geo g, int L) {
  extern __shared__ __align__(16) unsigned char per_smem[];
  T* tile = reinterpret_cast<T*>(per_smem);
  const PeriodicFam<T>& F = A.f[blockIdx.y];
  const int n = ZDIR ? g.nz : g.nx;
  const int ld = n + 1;
  const size_t P = (size_t)g.nz * g.nx;
  // the block's lines: x: rows row0 .. row0 + L - 1 of the family's planes;
  // z: columns i0 .. i0 + L - 1 of plane j
  const int blocks_per_plane = ZDIR ? g.nx / L : 0;
  const int nlines = ZDIR ? F.nplanes * (g.nx / L) : F.nplanes * g.nz / L;
  if ((int)blockIdx.x >= nlines) return;
  const int j = ZDIR ? blockIdx.x / blocks_per_plane : 0;
  const int i0 = ZDIR ? (blockIdx.x % blocks_per_plane) * L : 0;
  const size_t row0 = ZDIR ? 0 : (size_t)blockIdx.x * L;
  auto gidx = [&](int line, int pt) -> size_t {
    return ZDIR ? (size_t)j * P + (size_t)pt * g.nx + i0 + line : (row0 + line) * g.nx + pt;
  };
  const int tot = L * n;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int line = ZDIR ? e % L : e / n, pt = ZDIR ? e / L : e % n;
    tile[line * ld + pt] = F.r[gidx(line, pt)];
  }
  __syncthreads();
  if ((int)threadIdx.x < L) {
    T* x = tile + threadIdx.x * ld;
    T d = T(0);
    for (int i = 0; i < n; ++i) {
      d = (x[i] - (i ? F.lo * d : T(0))) * F.m[i];
      x[i] = d;
    }
    T y = d;   // y_{n-1} = d_{n-1}
    const T ylast = y;
    for (int i = n - 2; i >= 0; --i) {
      y = x[i] - F.cp[i] * y;
      x[i] = y;
    }
    const T f = (x[0] + F.log * ylast) * F.fac;
    for (int i = 0; i < n; ++i) x[i] -= f * F.q[i];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int line = ZDIR ? e % L : e / n, pt = ZDIR ? e / L : e % n;
    F.r[gidx(line, pt)] = tile[line * ld + pt];
  }
}

template <typename T>
cudaError_t launch_periodic(const PeriodicArgs<T>& a, const Geo& g, bool zdir, cudaStream_t s) {
  const int n = zdir ? g.nz : g.nx;
  int L = 32;
  while (L > 1 && (size_t)L * (n + 1) * sizeof(T) > 96 * 1024) L >>= 1;
  if (zdir && L > g.nx) L = g.nx;
  if (!zdir && L > g.nz) L = g.nz;
  const size_t smem = (size_t)L * (n + 1) * sizeof(T);
  int maxp = 0;
  for (int q = 0; q < a.nfam; ++q) maxp = a.f[q].nplanes > maxp ? a.f[q].nplanes : maxp;
  const int nblk = zdir ? maxp * (g.nx / L) : maxp * g.nz / L;
  auto kern = zdir ? k_periodic<T, true> : k_periodic<T, false>;
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<dim3((unsigned)nblk, (unsigned)a.nfam, 1), 128, smem, s>>>(a, g, L);
  return cudaGetLastError();
}

template cudaError_t launch_periodic<double>(const PeriodicArgs<double>&, const Geo&, bool, cudaStream_t);
template cudaError_t launch_periodic<float>(const PeriodicArgs<float>&, const Geo&, bool, cudaStream_t);

// ---------------------------------------------------------------------------
// Periodic x / z sweeps as truncated circulant convolutions, both directions in
// one pass.  Along x (and likewise z) every line of a family solves the same
// cyclic system (I - s L) with constant coefficients, whose inverse is
// circulant: x_i = sum_k g_k r_(i-k), g = (I - s L)^-1 e_0 symmetric and
// decaying like rho^|k|; the host keeps g_0 .. g_K.  The x and z operators act
// on different axes of a periodic tensor grid and commute, so one pass applies
// both.  A block owns one plane of one family; a thread owns V consecutive
// x-columns (one 16-byte vector).  The plane's rows (z) stream through a
// cp.async ring of kConvRing rows; each row is convolved along x from shared
// memory (KX taps: the thread's vector and its neighbours', periodic), and
// each thread convolves its columns along z in a register window of 2 KZ + 1
// rows.  The march reads rows nz - KZ .. nz - 1 (the window's start), then rows
// 0 .. nz - 1; the x-results of rows 0 .. KZ - 1 are kept in registers for the
// window's end.  Each output row is written after the last read of it, so the
// update is in place.
// ---------------------------------------------------------------------------
constexpr int kConvRing = 16;

template <typename T, int KX, int KZ>
__global__ void __launch_bounds__(512, 1) k_periodic_conv(ConvArgs<T> A, Geo g) {
  constexpr int V = 16 / sizeof(T);          // columns per thread
  constexpr int H = (KX + V - 1) / V;        // neighbouring vectors on each side
  using Vec = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
  extern __shared__ __align__(16) unsigned char conv_smem[];
  T* ring = reinterpret_cast<T*>(conv_smem);   // [kConvRing][nx]
  const ConvFam<T>& F = A.f[blockIdx.y];
  const int j = blockIdx.x;
  if (j >= F.nplanes) return;   // uniform per block: no barrier is skipped by part of it
  const int nx = g.nx, nz = g.nz, tid = threadIdx.x, nch = nx / V;
  T* base = F.r + (size_t)j * nz * nx;
  const int nseq = nz + KZ;
  auto row_of = [&](int s) { return (s + nz - KZ) & (nz - 1); };   // nz: a power of two
  auto issue = [&](int s) {   // one commit group per sequence index, empty past the end
    if (s < nseq) {
      const unsigned d = (unsigned)__cvta_generic_to_shared(ring + (size_t)(s % kConvRing) * nx + V * tid);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d),
                   "l"(base + (size_t)row_of(s) * nx + V * tid)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
#pragma unroll
  for (int s = 0; s < kConvRing - 1; ++s) issue(s);
  T gx[KX + 1], gz[KZ + 1];
#pragma unroll
  for (int t = 0; t <= KX; ++t) gx[t] = F.gx[t];
#pragma unroll
  for (int t = 0; t <= KZ; ++t) gz[t] = F.gz[t];
  T win[2 * KZ + 1][V], keep[KZ][V];
#pragma unroll
  for (int q = 0; q <= 2 * KZ; ++q)
#pragma unroll
    for (int o = 0; o < V; ++o) win[q][o] = T(0);
  // row s: wait for it, convolve it along x, push the result into the window
  auto row = [&](int s) {
    asm volatile("cp.async.wait_group %0;" ::"n"(kConvRing - 2) : "memory");   // row s: this thread's copy
    __syncthreads();   // every thread's copy of row s; every thread done with the slot of row s - 1
    issue(s + kConvRing - 1);
    const T* rw = ring + (size_t)(s % kConvRing) * nx;
    T v[(2 * H + 1) * V];
#pragma unroll
    for (int q = -H; q <= H; ++q) {
      const Vec w = *reinterpret_cast<const Vec*>(rw + V * ((tid + q) & (nch - 1)));
      const T* wp = reinterpret_cast<const T*>(&w);
#pragma unroll
      for (int o = 0; o < V; ++o) v[(q + H) * V + o] = wp[o];
    }
#pragma unroll
    for (int q = 0; q < 2 * KZ; ++q)
#pragma unroll
      for (int o = 0; o < V; ++o) win[q][o] = win[q + 1][o];
#pragma unroll
    for (int o = 0; o < V; ++o) {
      const int c = H * V + o;
      T xv = gx[0] * v[c];
#pragma unroll
      for (int t = 1; t <= KX; ++t) xv += gx[t] * (v[c - t] + v[c + t]);
      win[2 * KZ][o] = xv;
    }
  };
  // output row c from the window's centre
  auto store = [&](int c) {
    T y[V];
#pragma unroll
    for (int o = 0; o < V; ++o) {
      y[o] = gz[0] * win[KZ][o];
#pragma unroll
      for (int t = 1; t <= KZ; ++t) y[o] += gz[t] * (win[KZ - t][o] + win[KZ + t][o]);
    }
    *reinterpret_cast<Vec*>(base + (size_t)c * nx + V * tid) = *reinterpret_cast<const Vec*>(y);
  };
  for (int s = 0; s < 2 * KZ; ++s) {   // the window fills; rows 0 .. KZ - 1 are kept
    row(s);
#pragma unroll
    for (int q = 0; q < KZ; ++q)
      if (s == KZ + q)
#pragma unroll
        for (int o = 0; o < V; ++o) keep[q][o] = win[2 * KZ][o];
  }
  for (int s = 2 * KZ; s < nseq; ++s) {
    row(s);
    store(s - 2 * KZ);
  }
#pragma unroll
  for (int q = 0; q < KZ; ++q) {   // the window's end: rows 0 .. KZ - 1 again
#pragma unroll
    for (int p = 0; p < 2 * KZ; ++p)
#pragma unroll
      for (int o = 0; o < V; ++o) win[p][o] = win[p + 1][o];
#pragma unroll
    for (int o = 0; o < V; ++o) win[2 * KZ][o] = keep[q][o];
    store(nz - KZ + q);
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");   // no copy outlives the block
}

template <typename T>
cudaError_t launch_periodic_conv(const ConvArgs<T>& a, const Geo& g, cudaStream_t s) {
  constexpr int V = 16 / sizeof(T);
  const int nt = g.nx / V;
  if (g.nx % V || nt < 1 || nt > 512 || a.nfam < 1) return cudaErrorInvalidValue;
  if (a.kz != 2 && a.kz != 4 && a.kz != 8) return cudaErrorInvalidValue;
  if (2 * a.kz + 1 > g.nz) return cudaErrorInvalidValue;
  int kx = 0, maxp = 0;
  for (int q = 0; q < a.nfam; ++q) {
    kx = a.f[q].kx > kx ? a.f[q].kx : kx;
    maxp = a.f[q].nplanes > maxp ? a.f[q].nplanes : maxp;
  }
  const int KX = kx <= 4 ? 4 : 8;
  if (kx > kConvMaxK || 2 * KX + 1 > g.nx) return cudaErrorInvalidValue;
  if (maxp < 1) return cudaSuccess;
  const size_t smem = (size_t)kConvRing * g.nx * sizeof(T);
  const dim3 grd((unsigned)maxp, (unsigned)a.nfam);
  auto go = [&](auto kern) {
    if (smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    kern<<<grd, nt, smem, s>>>(a, g);
    return cudaGetLastError();
  };
  if (KX == 4) {
    switch (a.kz) {
      case 2: return go(k_periodic_conv<T, 4, 2>);
      case 4: return go(k_periodic_conv<T, 4, 4>);
      default: return go(k_periodic_conv<T, 4, 8>);
    }
  }
  switch (a.kz) {
    case 2: return go(k_periodic_conv<T, 8, 2>);
    case 4: return go(k_periodic_conv<T, 8, 4>);
    default: return go(k_periodic_conv<T, 8, 8>);
  }
}

template cudaError_t launch_periodic_conv<double>(const ConvArgs<double>&, const Geo&, cudaStream_t);
template cudaError_t launch_periodic_conv<float>(const ConvArgs<float>&, const Geo&, cudaStream_t);

template cudaError_t launch_cn_solves<double>(const Fields<double>&, const Geo&, const CNRows&, const CNRows&,
                                              const CNRows&, cudaStream_t);
template cudaError_t launch_cn_solves<float>(const Fields<float>&, const Geo&, const CNRows&, const CNRows&,
                                             const CNRows&, cudaStream_t);

template cudaError_t launch_fft_x_fwd<double, double>(PoissonSrc, const double*, const double*, const double*,
                                                      const double*, const double*, const double*, double,
                                                      const Geo&, const Metrics&, cplx<double>*,
                                                      const cplx<double>*, const cplx<double>*, cudaStream_t,
                                                      const float*, const float*, const double*, const float*,
                                                      const float*);
template cudaError_t launch_fft_x_fwd<float, float>(PoissonSrc, const float*, const float*, const float*,
                                                    const double*, const double*, const float*, double,
                                                    const Geo&, const Metrics&, cplx<float>*,
                                                    const cplx<float>*, const cplx<float>*, cudaStream_t,
                                                    const float*, const float*, const float*, const float*,
                                                    const float*);
template cudaError_t launch_fft_x_fwd<double, float>(PoissonSrc, const float*, const float*, const float*,
                                                     const double*, const double*, const double*, double,
                                                     const Geo&, const Metrics&, cplx<double>*,
                                                     const cplx<double>*, const cplx<double>*, cudaStream_t,
                                                     const float*, const float*, const double*, const float*,
                                                     const float*);

template cudaError_t launch_fft_z<double>(cplx<double>*, const cplx<double>*, const Geo&, bool, cudaStream_t);
template cudaError_t launch_fft_z<float>(cplx<float>*, const cplx<float>*, const Geo&, bool, cudaStream_t);

template cudaError_t launch_spec_thomas<double>(cplx<double>*, cplx<double>*, const double*, const double*,
                                                const YRows&, const Geo&, double, bool, cudaStream_t,
                                                const double*, const double*, double*);
template cudaError_t launch_spec_thomas<float>(cplx<float>*, cplx<double>*, const double*, const double*,
                                               const YRows&, const Geo&, double, bool, cudaStream_t,
                                               const double*, const double*, double*);

template cudaError_t launch_fft_x_inv<double, double>(PoissonDst, const cplx<double>*, const Geo&, const Metrics&,
                                                      const cplx<double>*, const cplx<double>*, double, double*,
                                                      cudaStream_t, const double*, const double*);
template cudaError_t launch_fft_x_inv<float, float>(PoissonDst, const cplx<float>*, const Geo&, const Metrics&,
                                                    const cplx<float>*, const cplx<float>*, double, float*,
                                                    cudaStream_t, const double*, const float*);
template cudaError_t launch_fft_x_inv<double, float>(PoissonDst, const cplx<double>*, const Geo&, const Metrics&,
                                                     const cplx<double>*, const cplx<double>*, double, float*,
                                                     cudaStream_t, const double*, const float*);

template cudaError_t launch_project<double>(double*, double*, double*, double*, const double*, double, bool,
                                            const Geo&, const double*, cudaStream_t);
template cudaError_t launch_project<float>(float*, float*, float*, float*, const float*, double, bool, const Geo&,
                                           const float*, cudaStream_t);

}  // namespace pnp
