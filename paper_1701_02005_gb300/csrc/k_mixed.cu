// Mixed-precision kernels of the fractional step (arXiv:1701.02005, Eqs. (1)-(4),
// Numerical methods; staggering of Fig. 1).
//
// Precision policy.  The parts that need FP64 accuracy keep a 48-bit or wider
// significand; on this GPU the per-cell ones get it from double-float pairs on
// the FP32 pipe (pnp_df.cuh), the 1-D ones from FP64:
//   * ion concentrations: an FP64 reference profile c_ref(y) plus a per-cell
//     double-float fluctuation (S, L), c = c_ref + S + L; S is the FP32 shadow
//     c' the stencils read;
//   * the potential: Phi = Phi_ref(y) + phi', phi' FP32 from the FP32 transform
//     of the fluctuating charge, its (0,0) mode from an FP64 source in FP64;
//   * every spectral y-solve in double-float (k_solve.cu);
//   * every product of two reference quantities (the 1-D double-layer
//     migration flux, its divergence, the implicit diffusion of c_ref and the
//     osmotic Coulomb force on v) is a per-plane FP64 constant folded in
//     exactly, so the near-cancellation of diffusion and migration inside the
//     Debye layer happens in FP64; only terms that contain a fluctuation are
//     rounded to FP32.
// c_ref, Phi_ref are plane means taken when the state is loaded.  Velocities,
// pressure and the momentum stencils are FP32; the velocity Crank-Nicolson
// matrix is I - s L_y with s L_y = O(1) (well conditioned) and runs in FP32.
#include "pnp_common.cuh"
#include "pnp_mixed.cuh"
#include "pnp_df.cuh"

namespace pnp {

// ---------------------------------------------------------------------------
// Ion Crank-Nicolson solve.  (I - s L_y) dc = Rref + r' is linear, so
// dc = dC_ref + (I - s L_y)^-1 r' with dC_ref the reference increment of the
// substage (a 1-D FP64 solve done on the host, passed as df pairs).  The
// fluctuation solve runs in FP32.  The ion state is the fluctuation about the
// fixed reference as a double-float pair, c = c_ref + S + L, so the shadow the
// stencils read is S itself; the update (S, L) += dC_ref + x' is df arithmetic
// on the FP32 pipe, with no FP64 instruction in the kernel.
// ---------------------------------------------------------------------------
__global__ void k_cn_ion_mixed(float* __restrict__ rcp, float* __restrict__ Sp, float* __restrict__ Lp,
                               float* __restrict__ rcm, float* __restrict__ Sm, float* __restrict__ Lm,
                               CNRowsF rows, const float2* __restrict__ dCp, const float2* __restrict__ dCm, int n,
                               size_t P) {
  constexpr int CH = 4;   // planes per batch; two batches in flight
  const size_t line = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= P) return;
  const bool plus = blockIdx.y == 0;
  float* r = plus ? rcp : rcm;
  float* S = plus ? Sp : Sm;
  float* L = plus ? Lp : Lm;
  const float2* dC = plus ? dCp : dCm;
  // forward sweep over batches [jb, jb + CH): the next batch's loads are
  // issued before this batch's recurrence
  auto load_f = [&](int jb, float (&rr)[CH]) {
#pragma unroll
    for (int u = 0; u < CH; ++u)
      if (jb + u < n) rr[u] = r[(size_t)(jb + u) * P + line];
  };
  auto comp_f = [&](int jb, const float (&rr)[CH], float d) {
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int j = jb + u;
      if (j < n) {
        d = (rr[u] - rows.a[j] * d) * rows.m[j];
        r[(size_t)j * P + line] = d;
      }
    }
    return d;
  };
  float d = 0.f;
  {
    float rA[CH], rB[CH];
    load_f(0, rA);
    for (int jb = 0; jb < n; jb += 2 * CH) {
      if (jb + CH < n) load_f(jb + CH, rB);
      d = comp_f(jb, rA, d);
      if (jb + CH < n) {
        if (jb + 2 * CH < n) load_f(jb + 2 * CH, rA);
        d = comp_f(jb + CH, rB, d);
      }
    }
  }
  // back substitution over batches jb, jb - 1, ..., jb - CH + 1, likewise
  auto load_b = [&](int jb, float (&dd)[CH], float (&sh)[CH], float (&sl)[CH]) {
#pragma unroll
    for (int u = 0; u < CH; ++u)
      if (jb - u >= 0) {
        const size_t o = (size_t)(jb - u) * P + line;
        dd[u] = r[o];
        sh[u] = S[o];
        sl[u] = L[o];
      }
  };
  auto comp_b = [&](int jb, const float (&dd)[CH], const float (&sh)[CH], const float (&sl)[CH], float x) {
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int j = jb - u;
      if (j >= 0) {
        const size_t o = (size_t)j * P + line;
        x = dd[u] - rows.c[j] * x;
        const float2 inc = dC[j];
        const dfl c = df_add2(dfl{sh[u], sl[u]}, dfl{inc.x, inc.y}, x);
        S[o] = c.h;
        L[o] = c.l;
      }
    }
    return x;
  };
  float x = 0.f;
  {
    float dA[CH], hA[CH], lA[CH], dB[CH], hB[CH], lB[CH];
    load_b(n - 1, dA, hA, lA);
    for (int jb = n - 1; jb >= 0; jb -= 2 * CH) {
      if (jb - CH >= 0) load_b(jb - CH, dB, hB, lB);
      x = comp_b(jb, dA, hA, lA, x);
      if (jb - CH >= 0) {
        if (jb - 2 * CH >= 0) load_b(jb - 2 * CH, dA, hA, lA);
        x = comp_b(jb - CH, dB, hB, lB, x);
      }
    }
  }
}

// FP32 velocity Crank-Nicolson solves (u, w: nyc cells; v: interior faces).
__global__ void k_cn_vel_f32(float* __restrict__ u, float* __restrict__ ru, float* __restrict__ v,
                             float* __restrict__ rv, float* __restrict__ w, float* __restrict__ rw,
                             CNRowsF cell, CNRowsF face, int nyc, size_t P) {
  constexpr int CH = 4;   // planes per batch; two batches in flight
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
  // both sweeps in CH-plane batches, the next batch's loads issued before this
  // batch's recurrence
  auto load_f = [&](int jb, float (&rr)[CH]) {
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (jb + k < n) rr[k] = rl[(size_t)(jb + k) * P];
  };
  auto comp_f = [&](int jb, const float (&rr)[CH], float d) {
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      const int j = jb + k;
      if (j < n) {
        d = (rr[k] - rw_.a[j] * d) * rw_.m[j];
        rl[(size_t)j * P] = d;
      }
    }
    return d;
  };
  float d = 0.f;
  {
    float rA[CH], rB[CH];
    load_f(0, rA);
    for (int jb = 0; jb < n; jb += 2 * CH) {
      if (jb + CH < n) load_f(jb + CH, rB);
      d = comp_f(jb, rA, d);
      if (jb + CH < n) {
        if (jb + 2 * CH < n) load_f(jb + 2 * CH, rA);
        d = comp_f(jb + CH, rB, d);
      }
    }
  }
  auto load_b = [&](int jb, float (&dd)[CH], float (&qq)[CH]) {
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (jb - k >= 0) {
        dd[k] = rl[(size_t)(jb - k) * P];
        qq[k] = ql[(size_t)(jb - k) * P];
      }
  };
  auto comp_b = [&](int jb, const float (&dd)[CH], const float (&qq)[CH], float x) {
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      const int j = jb - k;
      if (j >= 0) {
        x = dd[k] - rw_.c[j] * x;
        ql[(size_t)j * P] = qq[k] + x;
      }
    }
    return x;
  };
  float x = 0.f;
  {
    float dA[CH], qA[CH], dB[CH], qB[CH];
    load_b(n - 1, dA, qA);
    for (int jb = n - 1; jb >= 0; jb -= 2 * CH) {
      if (jb - CH >= 0) load_b(jb - CH, dB, qB);
      x = comp_b(jb, dA, qA, x);
      if (jb - CH >= 0) {
        if (jb - 2 * CH >= 0) load_b(jb - 2 * CH, dA, qA);
        x = comp_b(jb - CH, dB, qB, x);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Wall-normal CN solves with the right-hand sides in shared memory.  A block
// (one warp) owns 32 consecutive lines of one family.  The whole column block
// r[0..n)[32] arrives by 16-byte cp.async (every row in flight at once) and the
// forward elimination overwrites it with d in shared memory; the back
// substitution streams the state through a two-chunk ring of 16 planes (also
// cp.async, the first two chunks landing during the forward sweep) and writes
// it back with coalesced stores.  Against the line kernels above this drops
// the write and re-read of d in HBM (8 of the 20 / 28 bytes per cell of a
// velocity / ion family) and keeps ~7 warps' worth of rows in flight per SM.
// ---------------------------------------------------------------------------
struct CnFamily {
  const float* r;       // right-hand side at the family's first plane
  float* q0;            // state (velocity, or the high part S of an ion fluctuation)
  float* q1;            // low part L of an ion fluctuation (ion families)
  const float2* add;    // per-plane reference increment dC_ref (ion families)
  CNRowsF rows;
  int n;                // line length
};
struct CnTileArgs {
  CnFamily f[3];
  size_t P;
};

constexpr int kCnChunk = 16;   // planes per state chunk of the back substitution

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

// Shared memory (floats): d [n][32], state ring [2][NS][kCnChunk][32],
// factors a, m, c [n] each, then (ions) dC_ref [n] float2.
__host__ __device__ inline size_t cn_tile_floats(int n, int ns) {
  return (size_t)n * 32 + 2 * (size_t)ns * kCnChunk * 32 + 3 * (size_t)n + (n & 1) + (ns == 2 ? 2 * (size_t)n : 0);
}

// NS = state arrays per family: 1 (velocity) or 2 (ions, double-float update).
template <int NS>
__global__ void __launch_bounds__(32) k_cn_tile(CnTileArgs args) {
  extern __shared__ __align__(16) float cn_smem[];
  const CnFamily& F = args.f[blockIdx.y];
  const int n = F.n, t = threadIdx.x;
  const size_t P = args.P, line0 = (size_t)blockIdx.x * 32;
  float* sr = cn_smem;                                    // [n][32]: r, then d
  float* ring = sr + (size_t)n * 32;                      // [2][NS][kCnChunk][32]
  float* ca = ring + 2 * NS * kCnChunk * 32;              // [n] sub-diagonal factor a
  float* cm = ca + n;                                     // [n] 1 / pivot
  float* cc = cm + n;                                     // [n] c'
  float2* cadd = reinterpret_cast<float2*>(cc + n + (n & 1));   // [n] (ions)
  const int nchunks = (n + kCnChunk - 1) / kCnChunk;
  // chunk k of the back substitution: planes [hi - kCnChunk, hi), hi = n - k kCnChunk
  auto issue_chunk = [&](int k) {
    if (k < nchunks) {
      const int hi = n - k * kCnChunk, lo = max(0, hi - kCnChunk);
      float* buf = ring + (size_t)(k & 1) * NS * kCnChunk * 32;
      for (int e = t; e < (hi - lo) * 8; e += 32) {
        const int jj = e >> 3, c4 = (e & 7) * 4, j = hi - 1 - jj;
        cp_async16(buf + jj * 32 + c4, F.q0 + (size_t)j * P + line0 + c4);
        if constexpr (NS == 2) cp_async16(buf + kCnChunk * 32 + jj * 32 + c4, F.q1 + (size_t)j * P + line0 + c4);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  for (int e = t; e < n * 8; e += 32) {
    const int j = e >> 3, c4 = (e & 7) * 4;
    cp_async16(sr + j * 32 + c4, F.r + (size_t)j * P + line0 + c4);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  issue_chunk(0);
  issue_chunk(1);
  for (int j = t; j < n; j += 32) {
    ca[j] = F.rows.a[j];
    cm[j] = F.rows.m[j];
    cc[j] = F.rows.c[j];
    if constexpr (NS == 2) cadd[j] = F.add[j];
  }
  asm volatile("cp.async.wait_group 2;" ::: "memory");   // r has landed (this lane's copies)
  __syncwarp();                                         // ... and every lane's, with the factors
  float d = 0.f;
#pragma unroll 8
  for (int j = 0; j < n; ++j) {
    d = (sr[j * 32 + t] - ca[j] * d) * cm[j];
    sr[j * 32 + t] = d;
  }
  float x = 0.f;
  for (int k = 0; k < nchunks; ++k) {
    asm volatile("cp.async.wait_group 1;" ::: "memory");   // chunk k has landed
    __syncwarp();
    const float* buf = ring + (size_t)(k & 1) * NS * kCnChunk * 32;
    const int hi = n - k * kCnChunk, lo = max(0, hi - kCnChunk);
#pragma unroll 4
    for (int j = hi - 1; j >= lo; --j) {
      const int jj = hi - 1 - j;
      x = sr[j * 32 + t] - cc[j] * x;
      float* q0 = F.q0 + (size_t)j * P + line0 + t;
      if constexpr (NS == 1) {
        *q0 = buf[jj * 32 + t] + x;
      } else {
        const float2 inc = cadd[j];
        const dfl v = df_add2(dfl{buf[jj * 32 + t], buf[kCnChunk * 32 + jj * 32 + t]}, dfl{inc.x, inc.y}, x);
        *q0 = v.h;
        F.q1[(size_t)j * P + line0 + t] = v.l;
      }
    }
    __syncwarp();          // every lane is done with this buffer
    issue_chunk(k + 2);    // into the buffer just consumed
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

size_t cn_tile_smem(int n, int ns) { return sizeof(float) * cn_tile_floats(n, ns); }


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
  const double dp = cp[o] - R.cref64_p[j], dm = cm[o] - R.cref64_m[j];
  sh.cp[o] = (float)dp;
  sh.cpL[o] = (float)(dp - (double)sh.cp[o]);
  sh.cm[o] = (float)dm;
  sh.cmL[o] = (float)(dm - (double)sh.cm[o]);
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

// Ion concentration from its df fluctuation: c = c_ref(j) + S + L.
__global__ void k_from_shadow_df(const float* __restrict__ S, const float* __restrict__ L,
                                 const double* __restrict__ ref, double* __restrict__ out, size_t P, size_t n) {
  const size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  out[o] = ref[o / P] + ((double)S[o] + (double)L[o]);
}

// ---------------------------------------------------------------------------
cudaError_t launch_mixed_cn(const Fields<float>& f, const Shadows& sh, const MixedRefs& R, const Geo& g,
                            const CNRowsF& cell, const CNRowsF& face, const CNRowsF& ion, int l, unsigned parts,
                            cudaStream_t s) {
  const size_t P = (size_t)g.nz * g.nx;
  // lc_cn 32: shared-memory line tiles, when 32 lines divide a plane and a column
  // block fits; otherwise one thread per line, lc_cn threads per block (0: 128).
  // In the two-stream step the line kernels win (2.62 against 2.72 ms on the
  // 256x193x256 workload, although the tiles move 76 B per cell against 116 B
  // and are faster alone): the tiles' shared memory keeps the SMs from the
  // kernels of the other stream
  const bool tiled = g.lc_cn == 32 && P % 32 == 0 && cn_tile_smem(g.nyc, 2) <= 227 * 1024;
  if (tiled) {
    const dim3 blk(32);
    if (parts & kCnIons) {
      CnTileArgs a{};
      a.P = P;
      a.f[0] = CnFamily{reinterpret_cast<const float*>(f.rcp), sh.cp, sh.cpL, R.dC_p + (size_t)l * g.nyc, ion, g.nyc};
      a.f[1] = CnFamily{reinterpret_cast<const float*>(f.rcm), sh.cm, sh.cmL, R.dC_m + (size_t)l * g.nyc, ion, g.nyc};
      const size_t smem = cn_tile_smem(g.nyc, 2);
      if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_cn_tile<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
      }
      k_cn_tile<2><<<dim3((unsigned)(P / 32), 2), blk, smem, s>>>(a);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    if (parts & kCnVelocity) {
      CnTileArgs a{};
      a.P = P;
      a.f[0] = CnFamily{f.ru, f.u, nullptr, nullptr, cell, g.nyc};
      a.f[1] = CnFamily{f.rv + P, f.v + P, nullptr, nullptr, face, g.nyc - 1};   // interior faces 1 .. nyc-1
      a.f[2] = CnFamily{f.rw, f.w, nullptr, nullptr, cell, g.nyc};
      const size_t smem = cn_tile_smem(g.nyc, 1);
      if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_cn_tile<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
      }
      k_cn_tile<1><<<dim3((unsigned)(P / 32), 3), blk, smem, s>>>(a);
      return cudaGetLastError();
    }
    return cudaSuccess;
  }
  const int T = g.lc_cn > 32 ? g.lc_cn : 128;
  if (parts & kCnIons) {
    dim3 grd2((unsigned)((P + T - 1) / T), 2, 1);
    k_cn_ion_mixed<<<grd2, T, 0, s>>>(reinterpret_cast<float*>(f.rcp), sh.cp, sh.cpL,
                                      reinterpret_cast<float*>(f.rcm), sh.cm, sh.cmL, ion,
                                      R.dC_p + (size_t)l * g.nyc, R.dC_m + (size_t)l * g.nyc, g.nyc, P);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (parts & kCnVelocity) {
    dim3 grd((unsigned)((P + T - 1) / T), 3, 1);
    k_cn_vel_f32<<<grd, T, 0, s>>>(f.u, f.ru, f.v, f.rv, f.w, f.rw, cell, face, g.nyc, P);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Back substitution after the fused stencil (launch_mixed_rhs with CnFuse):
// the stencil stored, per y-chunk of its march, d~_j = (r_j - a_j d~_{j-1}) m_j
// started from zero at the chunk's first row, so the true forward value is
// d_j = d~_j + G_j d_{s-1}, G_j = prod_{i=s..j} (-a_i m_i) over the chunk
// (host table).  Per line: the chunk-end values d_{e-1} = d~_{e-1} + G_{e-1}
// d_{s-1} chunk by chunk (a few strided loads), then x_j = d_j - c_j x_{j+1}
// from the top, state += x (velocities; ions as the double-float update with
// the reference increment).  Reads d~ and the state once, writes the state.
// ---------------------------------------------------------------------------
struct FusedFam {
  const float* d;      // d~ at the family's first row
  float* S;            // state (velocity) or the high part S of an ion fluctuation
  float* L;            // low part L (ions), else nullptr
  const float2* add;   // dC_ref per row (ions), else nullptr
  const float* c;      // super-diagonal factor c per row
  const float* G;      // chunk products per row
  int n, j0;           // rows per line; plane of row 0
};
struct FusedArgs {
  FusedFam f[5];       // u, v, w, c+, c-
  int jc;
  size_t P;
};

template <bool ION>
__global__ void __launch_bounds__(256) k_cn_backsub_fused(FusedArgs A, int fam0) {
  constexpr int CH = 8;
  const FusedFam& F = A.f[fam0 + blockIdx.y];
  const size_t P = A.P;
  const size_t line = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= P) return;
  const int n = F.n, j0 = F.j0, jc = A.jc;
  const float* d = F.d + line;
  float* S = F.S + line;
  float* L = ION ? F.L + line : nullptr;
  // chunk ch holds rows [max(ch jc - j0, 0), min((ch + 1) jc - j0, n))
  const int nch = (n - 1 + j0) / jc + 1;
  float dend[kFusedMaxChunks];
  {
    float dv[kFusedMaxChunks];
#pragma unroll 8
    for (int ch = 0; ch < nch; ++ch) dv[ch] = d[(size_t)(min((ch + 1) * jc - j0, n) - 1) * P];
    float dp = 0.f;
    for (int ch = 0; ch < nch; ++ch) {
      dp = fmaf(F.G[min((ch + 1) * jc - j0, n) - 1], dp, dv[ch]);
      dend[ch] = dp;
    }
  }
  // back substitution from the top; the true d of the chunk below the current
  // row changes only when the sweep crosses into the next chunk down
  float x = 0.f;
  int ch = nch - 1;
  int first = max(ch * jc - j0, 0);
  float dprev = ch > 0 ? dend[ch - 1] : 0.f;
  for (int jb = n - 1; jb >= 0; jb -= CH) {
    float dd[CH], sh[CH], sl[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (jb - k >= 0) {
        const size_t o = (size_t)(jb - k) * P;
        dd[k] = d[o];
        sh[k] = S[o];
        if (ION) sl[k] = L[o];
      }
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      const int r = jb - k;
      if (r >= 0) {
        if (r < first) {
          --ch;
          first = max(ch * jc - j0, 0);
          dprev = ch > 0 ? dend[ch - 1] : 0.f;
        }
        x = fmaf(F.G[r], dprev, dd[k]) - F.c[r] * x;
        const size_t o = (size_t)r * P;
        if (ION) {
          const float2 inc = F.add[r];
          const dfl cv = df_add2(dfl{sh[k], sl[k]}, dfl{inc.x, inc.y}, x);
          S[o] = cv.h;
          L[o] = cv.l;
        } else {
          S[o] = sh[k] + x;
        }
      }
    }
  }
}

cudaError_t launch_mixed_cn_fused(const Fields<float>& f, const Shadows& sh, const MixedRefs& R, const Geo& g,
                                  const CNRowsF& cell, const CNRowsF& face, const CNRowsF& ion, const CnFusedG& G,
                                  int jc, int l, unsigned parts, cudaStream_t s) {
  const size_t P = (size_t)g.nz * g.nx;
  if ((g.nyc - 1) / jc + 1 > kFusedMaxChunks) return cudaErrorInvalidValue;
  FusedArgs A{};
  A.jc = jc;
  A.P = P;
  A.f[0] = FusedFam{f.ru, f.u, nullptr, nullptr, cell.c, G.cell, g.nyc, 0};
  A.f[1] = FusedFam{f.rv + P, f.v + P, nullptr, nullptr, face.c, G.face, g.nyc - 1, 1};
  A.f[2] = FusedFam{f.rw, f.w, nullptr, nullptr, cell.c, G.cell, g.nyc, 0};
  A.f[3] = FusedFam{reinterpret_cast<const float*>(f.rcp), sh.cp, sh.cpL, R.dC_p + (size_t)l * g.nyc, ion.c, G.ion,
                    g.nyc, 0};
  A.f[4] = FusedFam{reinterpret_cast<const float*>(f.rcm), sh.cm, sh.cmL, R.dC_m + (size_t)l * g.nyc, ion.c, G.ion,
                    g.nyc, 0};
  const int T = g.lc_cn && g.lc_cn != 32 ? g.lc_cn : 128;
  if (parts & kCnIons) {
    k_cn_backsub_fused<true><<<dim3((unsigned)((P + T - 1) / T), 2, 1), T, 0, s>>>(A, 3);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (parts & kCnVelocity) {
    k_cn_backsub_fused<false><<<dim3((unsigned)((P + T - 1) / T), 3, 1), T, 0, s>>>(A, 0);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// FP64-arithmetic variants of the mixed path's wall-normal CN solves (the
// "FP64 solves" policy): the FP32 right-hand sides are eliminated and
// back-substituted in FP64 with the FP64 factor rows, the forward values kept
// in FP64 scratch (d never rounds to FP32), and the update is added in FP64
// before the single rounding to the state's storage: velocities to FP32, the
// ion fluctuation (S, L) += dC_ref + x as an FP64 sum split back into a
// double-float pair.
// ---------------------------------------------------------------------------
template <int CH>
__device__ __forceinline__ double cn_forward_f64(const float* __restrict__ r, double* __restrict__ d_out,
                                                 const CNRows& rw, int n, size_t P) {
  double d = 0.0;
  for (int jb = 0; jb < n; jb += CH) {
    float rr[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u)
      if (jb + u < n) rr[u] = r[(size_t)(jb + u) * P];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int j = jb + u;
      if (j < n) {
        d = ((double)rr[u] - rw.a[j] * d) * rw.m[j];
        d_out[(size_t)j * P] = d;
      }
    }
  }
  return d;
}

__global__ void k_cn_vel_f64(float* __restrict__ u, const float* __restrict__ ru, float* __restrict__ v,
                             const float* __restrict__ rv, float* __restrict__ w, const float* __restrict__ rw,
                             double* __restrict__ du, double* __restrict__ dv, double* __restrict__ dw,
                             CNRows cell, CNRows face, int nyc, size_t P) {
  constexpr int CH = 8;
  const size_t line = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= P) return;
  float* q;
  const float* r;
  double* ds;
  CNRows rws;
  int n, j0;
  if (blockIdx.y == 0) { q = u; r = ru; ds = du; rws = cell; n = nyc; j0 = 0; }
  else if (blockIdx.y == 1) { q = v; r = rv; ds = dv; rws = face; n = nyc - 1; j0 = 1; }
  else { q = w; r = rw; ds = dw; rws = cell; n = nyc; j0 = 0; }
  const float* rl = r + (size_t)j0 * P + line;
  double* dl = ds + (size_t)j0 * P + line;
  float* ql = q + (size_t)j0 * P + line;
  cn_forward_f64<CH>(rl, dl, rws, n, P);
  double x = 0.0;
  for (int jb = n - 1; jb >= 0; jb -= CH) {
    double dd[CH];
    float qq[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (jb - k >= 0) {
        dd[k] = dl[(size_t)(jb - k) * P];
        qq[k] = ql[(size_t)(jb - k) * P];
      }
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      const int j = jb - k;
      if (j >= 0) {
        x = dd[k] - rws.c[j] * x;
        ql[(size_t)j * P] = (float)((double)qq[k] + x);
      }
    }
  }
}

__global__ void k_cn_ion_f64(const float* __restrict__ rcp, float* __restrict__ Sp, float* __restrict__ Lp,
                             const float* __restrict__ rcm, float* __restrict__ Sm, float* __restrict__ Lm,
                             double* __restrict__ dp, double* __restrict__ dm, CNRows rows,
                             const double* __restrict__ dCp, const double* __restrict__ dCm, int n, size_t P) {
  constexpr int CH = 8;
  const size_t line = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= P) return;
  const bool plus = blockIdx.y == 0;
  const float* r = (plus ? rcp : rcm) + line;
  float* S = (plus ? Sp : Sm) + line;
  float* L = (plus ? Lp : Lm) + line;
  double* dl = (plus ? dp : dm) + line;
  const double* dC = plus ? dCp : dCm;
  cn_forward_f64<CH>(r, dl, rows, n, P);
  double x = 0.0;
  for (int jb = n - 1; jb >= 0; jb -= CH) {
    double dd[CH];
    float sh[CH], sl[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (jb - k >= 0) {
        const size_t o = (size_t)(jb - k) * P;
        dd[k] = dl[o];
        sh[k] = S[o];
        sl[k] = L[o];
      }
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      const int j = jb - k;
      if (j >= 0) {
        const size_t o = (size_t)j * P;
        x = dd[k] - rows.c[j] * x;
        const double t = ((double)sh[k] + (double)sl[k]) + (dC[j] + x);
        const float hi = (float)t;
        S[o] = hi;
        L[o] = (float)(t - (double)hi);
      }
    }
  }
}

cudaError_t launch_mixed_cn_fp64(const Fields<float>& f, const Shadows& sh, const MixedRefs& R, const Geo& g,
                                 const CNRows& cell, const CNRows& face, const CNRows& ion, int l, unsigned parts,
                                 const CnScratch64& scr, cudaStream_t s) {
  const size_t P = (size_t)g.nz * g.nx;
  const int T = 128;
  if (parts & kCnIons) {
    dim3 grd((unsigned)((P + T - 1) / T), 2, 1);
    k_cn_ion_f64<<<grd, T, 0, s>>>(reinterpret_cast<const float*>(f.rcp), sh.cp, sh.cpL,
                                   reinterpret_cast<const float*>(f.rcm), sh.cm, sh.cmL, scr.dcp, scr.dcm, ion,
                                   R.Rref_p + (size_t)l * g.nyc, R.Rref_m + (size_t)l * g.nyc, g.nyc, P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (parts & kCnVelocity) {
    dim3 grd((unsigned)((P + T - 1) / T), 3, 1);
    k_cn_vel_f64<<<grd, T, 0, s>>>(f.u, f.ru, f.v, f.rv, f.w, f.rw, scr.du, scr.dv, scr.dw, cell, face, g.nyc, P);
    return cudaGetLastError();
  }
  return cudaSuccess;
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

cudaError_t launch_from_shadow_df(const float* S, const float* L, const double* ref, double* out, size_t P, size_t n,
                                  cudaStream_t s) {
  const int T = 256;
  k_from_shadow_df<<<(unsigned)((n + T - 1) / T), T, 0, s>>>(S, L, ref, out, P, n);
  return cudaGetLastError();
}

cudaError_t launch_from_shadow(const float* sh, const double* ref, double* out, size_t P, size_t n, cudaStream_t s) {
  const int T = 256;
  k_from_shadow<<<(unsigned)((n + T - 1) / T), T, 0, s>>>(sh, ref, out, P, n);
  return cudaGetLastError();
}

}  // namespace pnp
