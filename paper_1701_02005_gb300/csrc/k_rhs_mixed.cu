// Explicit right-hand sides of the mixed-precision fractional step
// (arXiv:1701.02005, Eqs. (1)-(3), Numerical methods; staggering of Fig. 1).
//
// FP32, one pass per cell: momentum (u, w on every cell; v on faces j >= 1),
// then both ions, reusing the loaded velocities and shadows.  For the ions the
// CN right-hand side is split as r_c = Rref(j) + r', Rref the per-plane FP64
// reference part (solved once per substage on the host and added by the ion
// CN update) and r' = dt [gam H' + zet H'_old + alp D L_y c'] stored in FP32.
//
// Both kernels march a chunk of y-planes per block and keep the seven stencil
// inputs (u, w, v, p, phi', c+', c-') of planes j-1, j, j+1 in a ring of plane
// slots in shared memory while the next planes land (four slots and one plane
// ahead for the TMA rows, five slots and two planes ahead for the tiles):
//   * k_rhs_mixed_tma: a block owns TZB full x-rows; each row of each array
//     arrives by one TMA tensor copy (cp.async.bulk.tensor, issued by one
//     warp, completion on an mbarrier per slot).  The z-halo rows are row
//     copies at the wrapped z, and after a plane lands its rows get a
//     one-float periodic x-halo from inside shared memory, so no copy ever
//     leaves the array.  nx in {32, 64, 128, 256}.
//   * k_rhs_mixed_tile: TX x TZ tiles with a one-cell periodic halo, filled by
//     per-thread cp.async (16-byte chunks for the rows, 4 bytes for the x-halo);
//     any grid.
// Tile geometry is compile-time in both, so every neighbour read is a
// shared-memory load at a constant offset from one of three slot pointers.
// The arithmetic of a cell is one routine (rhs_cell), specialised at compile
// time for interior planes and for the wall planes; the y-face products and
// ion fluxes at face j+1 are carried in registers to the next plane, where
// the same expression would be re-evaluated from the same operands.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <type_traits>

#include "pnp_common.cuh"
#include "pnp_mixed.cuh"

namespace pnp {

namespace {

constexpr int AU = 0, AW = 1, AV = 2, AP = 3, APH = 4, ACP = 5, ACM = 6, NA = 7, NH = 5;

// Per-plane constants of plane j (and of face j + 1 where a cell needs both faces).
struct PlaneC {
  float idy, ih, ihp, lo_c, hi_c, lo_f, hi_f, wl, wu;
  float rho_ref, Fvref, rhorf, dPref, dPrefp;
  float cref_p, cref_m, crf_p, crf_pp, crf_m, crf_mp;
  float Dih, Dihp;   // D / h_j, D / h_{j+1}
  // forward-elimination factors a, m of the CN rows at plane j (cells: u, w
  // and the ions; v: row j - 1, its face j), when the stencil eliminates
  float fa_c, fm_c, fa_f, fm_f, fa_i, fm_i;
};
constexpr int kPlaneC = 28;   // fields of PlaneC
constexpr int kPlaneLd = 28;  // table row length (16-byte rows)

// One field of PlaneC of plane j, by index.
__device__ __forceinline__ float plane_const(const MetricsF& mt, const MixedRefs& R, const CnFuse& fz, float D,
                                             int which, int j) {
  switch (which) {
    case 22: return fz.on ? fz.cell.a[j] : 0.f;
    case 23: return fz.on ? fz.cell.m[j] : 0.f;
    case 24: return fz.on && j > 0 ? fz.face.a[j - 1] : 0.f;
    case 25: return fz.on && j > 0 ? fz.face.m[j - 1] : 0.f;
    case 26: return fz.on ? fz.ion.a[j] : 0.f;
    case 27: return fz.on ? fz.ion.m[j] : 0.f;
    case 0: return mt.idy[j];
    case 1: return mt.ih[j];
    case 2: return mt.ih[j + 1];
    case 3: return mt.lo_c[j];
    case 4: return mt.hi_c[j];
    case 5: return mt.lo_f[j];
    case 6: return mt.hi_f[j];
    case 7: return mt.wl[j];
    case 8: return mt.wu[j];
    case 9: return R.rho_ref[j];
    case 10: return R.Fvref[j];
    case 11: return R.rhorf[j];
    case 12: return R.dPref[j];
    case 13: return R.dPref[j + 1];
    case 14: return R.cref_p[j];
    case 15: return R.cref_m[j];
    case 16: return R.crf_p[j];
    case 17: return R.crf_p[j + 1];
    case 18: return R.crf_m[j];
    case 19: return R.crf_m[j + 1];
    case 20: return D * mt.ih[j];
    default: return D * mt.ih[j + 1];
  }
}

// A block's table of per-plane constants: t[p * kPlaneLd + field], plane jb + p.
__device__ __forceinline__ void fill_plane_table(float* t, const MetricsF& mt, const MixedRefs& R, const CnFuse& fz,
                                                 float D, int jb, int je, int jchunk, int tid, int nthr) {
  for (int e = tid; e < kPlaneLd * jchunk; e += nthr) {
    const int p = e / kPlaneLd, which = e % kPlaneLd;
    t[e] = (which < kPlaneC && jb + p < je) ? plane_const(mt, R, fz, D, which, jb + p) : 0.f;
  }
}

__device__ __forceinline__ PlaneC plane_consts(const float* t) {
  PlaneC q;
  q.idy = t[0]; q.ih = t[1]; q.ihp = t[2];
  q.lo_c = t[3]; q.hi_c = t[4]; q.lo_f = t[5]; q.hi_f = t[6];
  q.wl = t[7]; q.wu = t[8];
  q.rho_ref = t[9]; q.Fvref = t[10]; q.rhorf = t[11]; q.dPref = t[12]; q.dPrefp = t[13];
  q.cref_p = t[14]; q.cref_m = t[15];
  q.crf_p = t[16]; q.crf_pp = t[17]; q.crf_m = t[18]; q.crf_mp = t[19];
  q.Dih = t[20]; q.Dihp = t[21];
  q.fa_c = t[22]; q.fm_c = t[23]; q.fa_f = t[24]; q.fm_f = t[25]; q.fa_i = t[26]; q.fm_i = t[27];
  return q;
}

// Two cells of one thread as a packed pair (cell 0 in .x, cell 1 in .y):
// arithmetic on the pair issues one packed FP32 instruction (FADD2 / FMUL2 /
// FFMA2) for both cells.  A float converts to the pair (both lanes).
struct V2 {
  float2 v;
  __device__ __forceinline__ V2() {}
  __device__ __forceinline__ V2(float a) : v(make_float2(a, a)) {}
  __device__ __forceinline__ V2(float a, float b) : v(make_float2(a, b)) {}
};
__device__ __forceinline__ V2 operator+(V2 a, V2 b) {
  V2 r;
  r.v = __fadd2_rn(a.v, b.v);
  return r;
}
__device__ __forceinline__ V2 operator-(V2 a, V2 b) {   // a + (-1) b: one rounding, as a - b
  V2 r;
  r.v = __ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v);
  return r;
}
__device__ __forceinline__ V2 operator*(V2 a, V2 b) {
  V2 r;
  r.v = __fmul2_rn(a.v, b.v);
  return r;
}
__device__ __forceinline__ V2 operator-(V2 a) { return V2(-a.v.x, -a.v.y); }
__device__ __forceinline__ V2 fmaT(V2 a, V2 b, V2 c) {
  V2 r;
  r.v = __ffma2_rn(a.v, b.v, c.v);
  return r;
}
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }

template <typename T>
struct CellOut {
  T ru, Hu, rw, Hw, rv, Hv, rcp, Hcp, rcm, Hcm;
};

// Values at face j+1 computed for plane j and reused as the face-j values of
// plane j+1: advective products of u, w, v and the ion fluxes.
template <typename T>
struct YCarry {
  T tu, tw, tv, fp, fm;
};

// Column wall velocities of the cell(s).
template <typename T>
struct CellK {
  T ub, ut, wb, wt;
};

// A tile value of the cell (T = float) or of the cell pair, the second cell one
// z-row (SZ floats) further (T = V2).
template <typename T, int SZ>
__device__ __forceinline__ T tld(const float* b, int i) {
  if constexpr (std::is_same<T, float>::value) return b[i];
  else return V2(b[i], b[i + SZ]);
}

// The FP32 explicit terms and CN right-hand sides of one cell or of a cell pair
// (and of the v-face below when DN).  bm, bo, bp: the (first) cell in array 0
// of the slots of planes j-1, j, j+1; arrays are AS floats apart, z-rows SZ
// floats apart.  DN / UP: a cell plane below / above exists; CIN: cy holds
// face j's values.  The products and sums are written as fused multiply-adds
// where a plain expression would let the compiler fuse them.
template <typename T, int AS, int SZ, bool DN, bool UP, bool CIN>
__device__ __forceinline__ CellOut<T> rhs_cell(const float* __restrict__ bm, const float* __restrict__ bo,
                                               const float* __restrict__ bp, const T Ho[5], const PlaneC& q,
                                               const CellK<T>& kw, const CoefF& k, YCarry<T>& cy) {
#define LM(a, off) tld<T, SZ>(bm, (a) * AS + (off))
#define LO(a, off) tld<T, SZ>(bo, (a) * AS + (off))
#define LP(a, off) tld<T, SZ>(bp, (a) * AS + (off))
  constexpr int XM = -1, XP = 1, ZM = -SZ, ZP = SZ;
  CellOut<T> o;
  const T u0 = LO(AU, 0), uxm = LO(AU, XM), uxp = LO(AU, XP), uzm = LO(AU, ZM), uzp = LO(AU, ZP);
  const T w0 = LO(AW, 0), wxm = LO(AW, XM), wxp = LO(AW, XP), wzm = LO(AW, ZM), wzp = LO(AW, ZP);
  const T vb = LO(AV, 0), vt = LP(AV, 0);
  const T p0 = LO(AP, 0);
  const T ph0 = LO(APH, 0), phxm = LO(APH, XM), phxp = LO(APH, XP), phzm = LO(APH, ZM), phzp = LO(APH, ZP);
  const T cp0 = LO(ACP, 0), cm0 = LO(ACM, 0);
  const T rho0 = cp0 - cm0;   // rho' at the centre
  const T dphxm = ph0 - phxm, dphxp = phxp - ph0, dphzm = ph0 - phzm, dphzp = phzp - ph0;
  T uym = 0.f, wym = 0.f, phym = 0.f, uyp = 0.f, wyp = 0.f, phyp = 0.f;
  if constexpr (DN) {
    uym = LM(AU, 0);
    wym = LM(AW, 0);
    phym = LM(APH, 0);
  }
  if constexpr (UP) {
    uyp = LP(AU, 0);
    wyp = LP(AW, 0);
    phyp = LP(APH, 0);
  }

  // u at (x-face i, y-centre j, z-centre k)
  {
    const T ubp = 0.5f * (u0 + uxp), ubm = 0.5f * (uxm + u0);
    const T ax = fmaT(ubp, ubp, -(ubm * ubm)) * k.idx;
    T ttop = 0.f, tbot = 0.f;
    if constexpr (UP) ttop = (0.5f * (LP(AV, XM) + vt)) * (0.5f * (u0 + uyp));
    if constexpr (DN) tbot = CIN ? cy.tu : (0.5f * (LO(AV, XM) + vb)) * (0.5f * (uym + u0));
    cy.tu = ttop;
    const T ay = (ttop - tbot) * q.idy;
    const T wfk = 0.5f * (wxm + w0);
    const T wfkp = 0.5f * (LO(AW, ZP + XM) + wzp);
    const T az = fmaT(wfkp, 0.5f * (u0 + uzp), -(wfk * (0.5f * (uzm + u0)))) * k.idz;
    const T lap = fmaT(fmaT(-2.f, u0, uzp) + uzm, k.idz2, (fmaT(-2.f, u0, uxp) + uxm) * k.idx2);
    const T rhom = LO(ACP, XM) - LO(ACM, XM);
    const T fu = (-k.Kx) * fmaT(0.5f, rhom + rho0, q.rho_ref) * dphxm;
    const T H = fmaT(k.nuH, lap, fu) - (ax + ay + az);
    const T Ly = fmaT(q.hi_c, (UP ? uyp : kw.ut) - u0, q.lo_c * ((DN ? uym : kw.ub) - u0));
    const T gp = (p0 - LO(AP, XM)) * k.idx;
    o.ru = k.dt * fmaT(k.anu, Ly, fmaT(k.anuxz, lap, fmaT(-k.alp, gp, fmaT(k.gam, H, k.zet * Ho[0]))));
    o.Hu = H;
  }
  // w at (x-centre i, y-centre j, z-face k)
  {
    const T wbp = 0.5f * (w0 + wzp), wbm = 0.5f * (wzm + w0);
    const T az = fmaT(wbp, wbp, -(wbm * wbm)) * k.idz;
    T ttop = 0.f, tbot = 0.f;
    if constexpr (UP) ttop = (0.5f * (LP(AV, ZM) + vt)) * (0.5f * (w0 + wyp));
    if constexpr (DN) tbot = CIN ? cy.tw : (0.5f * (LO(AV, ZM) + vb)) * (0.5f * (wym + w0));
    cy.tw = ttop;
    const T ay = (ttop - tbot) * q.idy;
    const T ufi = 0.5f * (uzm + u0);
    const T ufip = 0.5f * (LO(AU, ZM + XP) + uxp);
    const T ax = fmaT(ufip, 0.5f * (w0 + wxp), -(ufi * (0.5f * (wxm + w0)))) * k.idx;
    const T lap = fmaT(fmaT(-2.f, w0, wzp) + wzm, k.idz2, (fmaT(-2.f, w0, wxp) + wxm) * k.idx2);
    const T rhom = LO(ACP, ZM) - LO(ACM, ZM);
    const T fw = (-k.Kz) * fmaT(0.5f, rhom + rho0, q.rho_ref) * dphzm;
    const T H = fmaT(k.nuH, lap, fw) - (ax + ay + az);
    const T Ly = fmaT(q.hi_c, (UP ? wyp : kw.wt) - w0, q.lo_c * ((DN ? wym : kw.wb) - w0));
    const T gp = (p0 - LO(AP, ZM)) * k.idz;
    o.rw = k.dt * fmaT(k.anu, Ly, fmaT(k.anuxz, lap, fmaT(-k.alp, gp, fmaT(k.gam, H, k.zet * Ho[1]))));
    o.Hw = H;
  }
  // v at (x-centre i, y-face j, z-centre k), 1 <= j <= nyc-1; the centre
  // product (v_j + v_j+1)^2 / 4 is the face-j product of the next plane
  {
    const T vbu = 0.5f * (vb + vt);
    const T ttop = vbu * vbu;
    o.rv = 0.f;
    o.Hv = 0.f;
    if constexpr (DN) {
      const T v0 = vb;
      const T vxm = LO(AV, XM), vxp = LO(AV, XP), vzm = LO(AV, ZM), vzp = LO(AV, ZP);
      const T vym = LM(AV, 0), vyp = vt;
      T tbot;
      if constexpr (CIN) {
        tbot = cy.tv;
      } else {
        const T vbd = 0.5f * (vym + v0);
        tbot = vbd * vbd;
      }
      const T Ui = fmaT(q.wl, uym, q.wu * u0);
      const T Uip = fmaT(q.wl, LM(AU, XP), q.wu * uxp);
      const T ax = fmaT(Uip, 0.5f * (v0 + vxp), -(Ui * (0.5f * (vxm + v0)))) * k.idx;
      const T ay = (ttop - tbot) * q.ih;
      const T Wk = fmaT(q.wl, wym, q.wu * w0);
      const T Wkp = fmaT(q.wl, LM(AW, ZP), q.wu * wzp);
      const T az = fmaT(Wkp, 0.5f * (v0 + vzp), -(Wk * (0.5f * (vzm + v0)))) * k.idz;
      const T lap = fmaT(fmaT(-2.f, v0, vzp) + vzm, k.idz2, (fmaT(-2.f, v0, vxp) + vxm) * k.idx2);
      // Coulomb force: reference-reference part is the FP64 constant Fvref
      const T rhod = LM(ACP, 0) - LM(ACM, 0);
      const T rpf = 0.5f * (rhod + rho0);   // rho' on the face
      const T dphi = ph0 - phym;            // phi' difference
      const T fv = fmaT(-k.K * q.ih, fmaT(q.rhorf, dphi, rpf * (dphi + q.dPref)), q.Fvref);
      const T H = fmaT(k.nuH, lap, fv) - (ax + ay + az);
      const T Ly = fmaT(q.hi_f, vyp - v0, q.lo_f * (vym - v0));
      const T gp = (p0 - LM(AP, 0)) * q.ih;
      o.rv = k.dt * fmaT(k.anu, Ly, fmaT(k.anuxz, lap, fmaT(-k.alp, gp, fmaT(k.gam, H, k.zet * Ho[2]))));
      o.Hv = H;
    }
    cy.tv = ttop;
  }
  // ions: FP32 fluctuation fluxes (the reference-reference part is in Rref);
  // F = c_face u - D (dc/dn + s c_face dphi/dn), D/dn folded into one factor
#pragma unroll
  for (int ion = 0; ion < 2; ++ion) {
    const int A = ion == 0 ? ACP : ACM;
    const float cr = ion == 0 ? q.cref_p : q.cref_m;
    const float sD = ion == 0 ? 1.f : -1.f;
    const T cc = ion == 0 ? cp0 : cm0;
    const T cxm_ = LO(A, XM), cxp_ = LO(A, XP), czm_ = LO(A, ZM), czp_ = LO(A, ZP);
    T ca = fmaT(0.5f, cxm_ + cc, cr), cb = fmaT(0.5f, cc + cxp_, cr);
    const T sca = ion == 0 ? ca : -ca, scb = ion == 0 ? cb : -cb;
    const T Fx_i = fmaT(u0, ca, (-k.Dx) * fmaT(sca, dphxm, cc - cxm_));
    const T Fx_ip = fmaT(uxp, cb, (-k.Dx) * fmaT(scb, dphxp, cxp_ - cc));
    ca = fmaT(0.5f, czm_ + cc, cr);
    cb = fmaT(0.5f, cc + czp_, cr);
    const T sza = ion == 0 ? ca : -ca, szb = ion == 0 ? cb : -cb;
    const T Fz_k = fmaT(w0, ca, (-k.Dz) * fmaT(sza, dphzm, cc - czm_));
    const T Fz_kp = fmaT(wzp, cb, (-k.Dz) * fmaT(szb, dphzp, czp_ - cc));
    // y faces: advection + migration
    T Fy_j = 0.f, Fy_jp = 0.f, Ly = 0.f;
    if constexpr (DN) {
      const T cym_ = LM(A, 0);
      Ly = q.lo_c * (cym_ - cc);
      if constexpr (CIN) {
        Fy_j = ion == 0 ? cy.fp : cy.fm;
      } else {
        const float crf = ion == 0 ? q.crf_p : q.crf_m;
        const T cpf = 0.5f * (cym_ + cc), dph = ph0 - phym;
        Fy_j = fmaT(vb, cpf + crf, (-sD * q.Dih) * fmaT(cpf, dph + q.dPref, crf * dph));
      }
    }
    if constexpr (UP) {
      const T cyp_ = LP(A, 0);
      Ly = fmaT(q.hi_c, cyp_ - cc, Ly);
      const float crfp = ion == 0 ? q.crf_pp : q.crf_mp;
      const T cpf = 0.5f * (cc + cyp_), dph = phyp - ph0;
      Fy_jp = fmaT(vt, cpf + crfp, (-sD * q.Dihp) * fmaT(cpf, dph + q.dPrefp, crfp * dph));
    }
    if (ion == 0) cy.fp = Fy_jp;
    else cy.fm = Fy_jp;
    const T div = fmaT(Fz_kp - Fz_k, k.idz, fmaT(Fy_jp - Fy_j, q.idy, (Fx_ip - Fx_i) * k.idx));
    T H = -div;
    T r = k.dt * fmaT(k.aD, Ly, fmaT(-k.gam, div, k.zet * Ho[3 + ion]));
    if (k.af) {   // the x/z diffusion leaves H and joins the implicit operator: r gains dt (alp - gam) D lap
      const T lapc = fmaT(fmaT(-2.f, cc, czp_) + czm_, k.idz2, (fmaT(-2.f, cc, cxp_) + cxm_) * k.idx2);
      H = fmaT(-k.D, lapc, H);
      r = fmaT(k.dt * k.zD, lapc, r);
    }
    if (ion == 0) {
      o.rcp = r;
      o.Hcp = H;
    } else {
      o.rcm = r;
      o.Hcm = H;
    }
  }
  return o;
#undef LM
#undef LO
#undef LP
}

// Plane j of a chunk starting at jb: the specialisation for its position.
template <typename T, int AS, int SZ>
__device__ __forceinline__ CellOut<T> rhs_cell_at(int j, int jb, int nyc, const float* bm, const float* bo,
                                                  const float* bp, const T Ho[5], const PlaneC& q,
                                                  const CellK<T>& kw, const CoefF& k, YCarry<T>& cy) {
  if (j > jb) {
    if (j < nyc - 1) return rhs_cell<T, AS, SZ, true, true, true>(bm, bo, bp, Ho, q, kw, k, cy);
    return rhs_cell<T, AS, SZ, true, false, true>(bm, bo, bp, Ho, q, kw, k, cy);
  }
  if (j > 0) {
    if (j < nyc - 1) return rhs_cell<T, AS, SZ, true, true, false>(bm, bo, bp, Ho, q, kw, k, cy);
    return rhs_cell<T, AS, SZ, true, false, false>(bm, bo, bp, Ho, q, kw, k, cy);
  }
  if (j < nyc - 1) return rhs_cell<T, AS, SZ, false, true, false>(bm, bo, bp, Ho, q, kw, k, cy);
  return rhs_cell<T, AS, SZ, false, false, false>(bm, bo, bp, Ho, q, kw, k, cy);
}

__device__ __forceinline__ void store_cell(const Fields<float>& f, float* rcp, float* rcm, const Shadows& sh,
                                           size_t c0, bool has_dn, bool keep_h, const CellOut<float>& o) {
  f.ru[c0] = o.ru;
  f.rw[c0] = o.rw;
  if (has_dn) f.rv[c0] = o.rv;
  rcp[c0] = o.rcp;
  rcm[c0] = o.rcm;
  if (keep_h) {
    f.Hu[c0] = o.Hu;
    f.Hw[c0] = o.Hw;
    if (has_dn) f.Hv[c0] = o.Hv;
    sh.Hcp[c0] = o.Hcp;
    sh.Hcm[c0] = o.Hcm;
  }
}

// The pair: cell 0 at c0, cell 1 at c1.
__device__ __forceinline__ void store_cell(const Fields<float>& f, float* rcp, float* rcm, const Shadows& sh,
                                           size_t c0, size_t c1, bool has_dn, bool keep_h, const CellOut<V2>& o) {
  f.ru[c0] = o.ru.v.x;
  f.ru[c1] = o.ru.v.y;
  f.rw[c0] = o.rw.v.x;
  f.rw[c1] = o.rw.v.y;
  if (has_dn) {
    f.rv[c0] = o.rv.v.x;
    f.rv[c1] = o.rv.v.y;
  }
  rcp[c0] = o.rcp.v.x;
  rcp[c1] = o.rcp.v.y;
  rcm[c0] = o.rcm.v.x;
  rcm[c1] = o.rcm.v.y;
  if (keep_h) {
    f.Hu[c0] = o.Hu.v.x;
    f.Hu[c1] = o.Hu.v.y;
    f.Hw[c0] = o.Hw.v.x;
    f.Hw[c1] = o.Hw.v.y;
    if (has_dn) {
      f.Hv[c0] = o.Hv.v.x;
      f.Hv[c1] = o.Hv.v.y;
    }
    sh.Hcp[c0] = o.Hcp.v.x;
    sh.Hcp[c1] = o.Hcp.v.y;
    sh.Hcm[c0] = o.Hcm.v.x;
    sh.Hcm[c1] = o.Hcm.v.y;
  }
}

// The CN forward elimination fused into the stencil: the right-hand sides of
// plane j become d~_j = (r_j - a_j d~_{j-1}) m_j, started from d~ = 0 at the
// chunk's first plane (the first v face for v), so each chunk of the y-march is
// an independent affine piece d_j = d~_j + G_j d_{s-1} of the line's true
// elimination; the CN back substitution supplies d_{s-1} (G_j: products of
// -a m over the chunk up to j, host tables).
template <typename T>
struct FwdCarry {
  T u, w, v, cp, cm;
};

template <typename T>
__device__ __forceinline__ void fuse_forward(CellOut<T>& o, const PlaneC& q, int j, int jb, FwdCarry<T>& d) {
  if (j == jb) d = FwdCarry<T>{0.f, 0.f, 0.f, 0.f, 0.f};
  d.u = fmaT(-q.fa_c, d.u, o.ru) * q.fm_c;
  d.w = fmaT(-q.fa_c, d.w, o.rw) * q.fm_c;
  if (j > 0) d.v = fmaT(-q.fa_f, d.v, o.rv) * q.fm_f;
  d.cp = fmaT(-q.fa_i, d.cp, o.rcp) * q.fm_i;
  d.cm = fmaT(-q.fa_i, d.cm, o.rcm) * q.fm_i;
  o.ru = d.u;
  o.rw = d.w;
  o.rv = d.v;
  o.rcp = d.cp;
  o.rcm = d.cm;
}

__device__ __forceinline__ void wall_values(const Fields<float>& f, size_t P, size_t ck, float Uw, float& ub,
                                            float& ut, float& wb, float& wt) {
  ub = f.wall_u ? f.wall_u[ck] : -Uw;
  ut = f.wall_u ? f.wall_u[P + ck] : Uw;
  wb = f.wall_w ? f.wall_w[ck] : 0.f;
  wt = f.wall_w ? f.wall_w[P + ck] : 0.f;
}

// ---------------------------------------------------------------------------
// cp.async tile kernel (any grid)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_but_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

// Tile geometry in shared memory.  A tile row holds the TX cells of one z-row
// from column 0 (16-byte aligned, so the interior lands by 16-byte copies), the
// +x halo at column TX and the -x halo of the NEXT row at column RS - 1; the
// array starts with a 4-float pad that holds row 0's -x halo.  Neighbours are
// therefore at -1 / +1 (x) and -RS / +RS (z) from every cell.
template <int TX, int TZ, int CZ>
struct TileGeo {
  static constexpr int PAD = 4, RS = TX + 4, ROWS = TZ * CZ + 2;
  static constexpr int NT = PAD + ROWS * RS;   // floats per array, a multiple of 4
  static constexpr int QX = TX / 4;            // 16-byte chunks per row
  static constexpr int TASKS = ROWS * (QX + 2);   // copies per array and plane
  static_assert(TX % 4 == 0, "16-byte interior copies");
};

// Plane ring: NSLOT slots, planes j-1, j, j+1 read while j+2 and j+3 land.
constexpr int kTileSlots = 5, kHoldSlots = 4;

// Shared memory of the tile kernel (floats): tiles [kTileSlots][7 arrays][NT],
// then (HSM) old H [kHoldSlots][5 arrays][CZ][TX TZ], then the per-plane
// table [jchunk][kPlaneLd].
__host__ __device__ constexpr size_t rhs_tile_floats(int tx, int tz, int cz, bool hsm) {
  return (size_t)kTileSlots * 7 * (4 + (size_t)(tz * cz + 2) * (tx + 4)) +
         (hsm ? (size_t)kHoldSlots * 5 * tx * tz * cz : 0);
}

// TX x TZ threads own a TX x (TZ CZ) tile of cells; each thread computes CZ
// cells stacked in z.  HSM: the previous substage's H arrives by cp.async with
// the planes (else each thread loads it at the top of the iteration).
//
// One barrier per plane: after it every thread has finished the previous
// plane, so the slot of plane j-2 is free for plane j+3, which is issued right
// behind the barrier and has two plane times to land.
template <int TX, int TZ, int CZ, bool HSM, int MINB>
__global__ void __launch_bounds__(TX * TZ, MINB)
    k_rhs_mixed_tile(Fields<float> f, float* __restrict__ rcp, float* __restrict__ rcm, Shadows sh, MixedRefs R,
                     Geo g, MetricsF mt, CoefF cf, int jchunk, CnFuse fz) {
  using TG = TileGeo<TX, TZ, CZ>;
  constexpr int NT = TG::NT, RS = TG::RS, NTH = TX * TZ, E = (TG::TASKS + NTH - 1) / NTH;
  extern __shared__ __align__(16) float rhs_smem[];
  float* tiles = rhs_smem;                                          // [kTileSlots][NA][NT]
  float* holds = rhs_smem + (size_t)kTileSlots * NA * NT;            // [kHoldSlots][NH][CZ][NTH] (HSM)
  float* pct = rhs_smem + rhs_tile_floats(TX, TZ, CZ, HSM);         // [jchunk][kPlaneLd]
  const int tx = threadIdx.x, tz = threadIdx.y, tid = tz * TX + tx;
  const int nx = g.nx, nz = g.nz, nyc = g.nyc;
  const int i0 = blockIdx.x * TX, k0 = blockIdx.y * (TZ * CZ);
  const int jb = blockIdx.z * jchunk, je = min(nyc, jb + jchunk);
  const size_t P = (size_t)nz * nx;
  // in-plane offset of this thread's first cell; the others are nx apart
  const size_t ck = (size_t)(k0 + tz * CZ) * nx + i0 + tx;

  // this thread's copies of every array's tile: task t < ROWS QX is the 16-byte
  // chunk t % QX of row t / QX; the next 2 ROWS tasks are the x-halo floats
  // (periodic in x and z); kind 16 / 4 bytes, 0 = none
  int goff[E], soff[E], kind[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int t = tid + e * NTH;
    kind[e] = 0;
    goff[e] = 0;
    soff[e] = 0;
    if (t < TG::ROWS * TG::QX) {
      const int r = t / TG::QX, qx = t % TG::QX;
      goff[e] = ((k0 - 1 + r) & (nz - 1)) * nx + i0 + 4 * qx;
      soff[e] = TG::PAD + r * RS + 4 * qx;
      kind[e] = 16;
    } else if (t < TG::TASKS) {
      const int h = t - TG::ROWS * TG::QX, r = h >> 1, side = h & 1;
      goff[e] = ((k0 - 1 + r) & (nz - 1)) * nx + ((side ? i0 + TX : i0 - 1) & (nx - 1));
      soff[e] = TG::PAD + r * RS + (side ? TX : -1);
      kind[e] = 4;
    }
  }
  const float* src[NA] = {f.u, f.w, f.v, f.p, sh.phi, sh.cp, sh.cm};
  const float* hsrc[NH] = {f.Hu, f.Hw, f.Hv, sh.Hcp, sh.Hcm};
  const bool read_h = cf.zet != 0.f, keep_h = cf.keep_h != 0;   // uniform per launch
  // ring position of plane q (q >= jb - 1)
  auto slot_of = [&](int q) { return (q - jb + 1) % kTileSlots; };
  // plane q (tiles into its slot, old H into slot (q - jb + 1) & 3); one commit
  // group per plane, empty when q is outside the chunk's window or the array
  auto issue_plane = [&](int q) {
    if (q >= jb - 1 && q <= je) {
      float* ts = tiles + (size_t)slot_of(q) * NA * NT;
      const size_t qP = (size_t)q * P;
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        if (q < 0 || q >= (a == AV ? nyc + 1 : nyc)) continue;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if (kind[e] == 16) cp_async16(ts + a * NT + soff[e], src[a] + qP + goff[e]);
          else if (kind[e] == 4) cp_async4(ts + a * NT + soff[e], src[a] + qP + goff[e]);
        }
      }
      if constexpr (HSM) {
        if (read_h && q >= jb && q < je) {
          float* hs = holds + (size_t)((q - jb + 1) & (kHoldSlots - 1)) * NH * CZ * NTH;
#pragma unroll
          for (int h = 0; h < NH; ++h)
#pragma unroll
            for (int cz = 0; cz < CZ; ++cz)
              cp_async4(hs + (h * CZ + cz) * NTH + tid, hsrc[h] + qP + ck + (size_t)cz * nx);
        }
      }
    }
    cp_async_commit();
  };
  issue_plane(jb - 1);
  issue_plane(jb);
  issue_plane(jb + 1);
  issue_plane(jb + 2);
  fill_plane_table(pct, mt, R, fz, cf.D, jb, je, jchunk, tid, NTH);
  const bool fuse = fz.on != 0;   // uniform per launch

  // CZ = 1: one cell in FP32 scalars; CZ = 2: the cell pair in packed FP32
  using T = typename std::conditional<CZ == 2, V2, float>::type;
  static_assert(CZ == 1 || CZ == 2, "one cell or a packed pair per thread");
  // wall velocities of the column(s), read only on the two wall planes
  auto walls = [&]() {
    float ub[CZ], ut[CZ], wb[CZ], wt[CZ];
#pragma unroll
    for (int cz = 0; cz < CZ; ++cz) wall_values(f, P, ck + (size_t)cz * nx, cf.Uw, ub[cz], ut[cz], wb[cz], wt[cz]);
    if constexpr (CZ == 2) return CellK<T>{V2(ub[0], ub[1]), V2(ut[0], ut[1]), V2(wb[0], wb[1]), V2(wt[0], wt[1])};
    else return CellK<T>{ub[0], ut[0], wb[0], wt[0]};
  };
  const int c = TG::PAD + (tz * CZ + 1) * RS + tx;   // first cell in a tile
  YCarry<T> cy{0.f, 0.f, 0.f, 0.f, 0.f};
  FwdCarry<T> fd{0.f, 0.f, 0.f, 0.f, 0.f};
  for (int j = jb; j < je; ++j) {
    const size_t c0 = (size_t)j * P + ck;
    float Hf[CZ][NH];
#pragma unroll
    for (int cz = 0; cz < CZ; ++cz)
#pragma unroll
      for (int h = 0; h < NH; ++h) Hf[cz][h] = 0.f;
    if constexpr (!HSM) {
      if (read_h) {
#pragma unroll
        for (int cz = 0; cz < CZ; ++cz) {
          const size_t o = c0 + (size_t)cz * nx;
#pragma unroll
          for (int h = 0; h < NH; ++h) Hf[cz][h] = __ldg(hsrc[h] + o);
        }
      }
    }
    cp_async_wait_all_but_one();   // planes up to j + 1 have landed (this thread's copies)
    __syncthreads();               // ... every thread's; and every thread is done with plane j - 2
    issue_plane(j + 3);            // into the slot of plane j - 2
    if constexpr (HSM) {
      if (read_h) {
        const float* hs = holds + (size_t)((j - jb + 1) & (kHoldSlots - 1)) * NH * CZ * NTH + tid;
#pragma unroll
        for (int h = 0; h < NH; ++h)
#pragma unroll
          for (int cz = 0; cz < CZ; ++cz) Hf[cz][h] = hs[(h * CZ + cz) * NTH];
      }
    }
    T Ho[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      if constexpr (CZ == 2) Ho[h] = V2(Hf[0][h], Hf[1][h]);
      else Ho[h] = Hf[0][h];
    }
    const float* bm = tiles + (size_t)slot_of(j - 1) * NA * NT + c;
    const float* bo = tiles + (size_t)slot_of(j) * NA * NT + c;
    const float* bp = tiles + (size_t)slot_of(j + 1) * NA * NT + c;
    const PlaneC q = plane_consts(pct + (size_t)(j - jb) * kPlaneLd);
    const CellK<T> kc = (j == 0 || j == nyc - 1) ? walls() : CellK<T>{0.f, 0.f, 0.f, 0.f};
    CellOut<T> o = rhs_cell_at<T, NT, RS>(j, jb, nyc, bm, bo, bp, Ho, q, kc, cf, cy);
    if (fuse) fuse_forward(o, q, j, jb, fd);
    if constexpr (CZ == 2) store_cell(f, rcp, rcm, sh, c0, c0 + nx, j > 0, keep_h, o);
    else store_cell(f, rcp, rcm, sh, c0, j > 0, keep_h, o);
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");   // no copy outlives the block
}

// ---------------------------------------------------------------------------
// TMA row kernel
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned sm_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_addr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sm_addr(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(sm_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for a phase of an mbarrier: gives up after limit_ns (two
// seconds for the stencil's copies) or 2^26 polls, so a copy that never
// completes cannot hang the GPU; the caller records the failure.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity,
                                          unsigned long long limit_ns = 2000000000ull) {
  if (mbar_try_wait(b, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (int it = 0; it < (1 << 26); ++it) {
    if (mbar_try_wait(b, parity)) return true;
    if ((it & 255) == 0 && global_ns() - t0 > limit_ns) break;
  }
  return false;
}

// Self-test of the failure path: one thread promises 16 bytes on an mbarrier
// that no copy ever completes and waits with the bounded wait above; the wait
// runs out and the timeout is recorded in the context's error word.  Nothing
// is in flight when the block exits.
__global__ void k_wait_selftest(int* __restrict__ err, unsigned long long limit_ns) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_arrive_expect_tx(&bar, 16);
    if (!mbar_wait(&bar, 0, limit_ns)) atomicExch(err, PNP_ERR_TIMEOUT);
  }
}

__device__ __forceinline__ void tma_row(float* dst, const CUtensorMap* m, int x, int z, int y,
                                        unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(sm_addr(dst)),
      "l"(reinterpret_cast<unsigned long long>(m)), "r"(x), "r"(z), "r"(y), "r"(sm_addr(bar))
      : "memory");
}

// Geometry of the TMA kernel for nx = NX, TZB rows per block:
//   row stride S = NX + 32 floats: row data at [32, 32 + NX) (128-byte aligned
//   for the TMA destination), x-halo at 31 and 32 + NX (= 0 of the next row);
//   an array-slot region holds TZB + 2 rows (z = k0-1 .. k0+TZB, wrapped) plus
//   the last row's right halo.  Then old H [4 slots][5][TZB][NX], the
//   per-plane table [jchunk][kPlaneLd] and four 8-byte mbarriers.
template <int NX, int TZB>
struct TmaGeo {
  static constexpr int S = NX + 32, ROWS = TZB + 2, AS = ROWS * S + 32, SLOT = NA * AS;
  static constexpr int BW = NX < 256 ? NX : 256, NBOX = NX / BW;
  static constexpr int HS = NH * TZB * NX;   // old-H slot
  static constexpr int NTHR = NX * TZB;
  static constexpr size_t floats(int jchunk) { return 4 * (size_t)SLOT + 4 * (size_t)HS + (size_t)kPlaneLd * jchunk; }
  static constexpr size_t bytes(int jchunk) { return floats(jchunk) * sizeof(float) + 4 * sizeof(unsigned long long); }
};

template <int NX, int TZB>
__global__ void __launch_bounds__(NX * TZB, 1)
    k_rhs_mixed_tma(const __grid_constant__ RhsMaps maps, Fields<float> f, float* __restrict__ rcp,
                    float* __restrict__ rcm, Shadows sh, MixedRefs R, Geo g, MetricsF mt, CoefF cf, int jchunk,
                    int* __restrict__ err, CnFuse fz) {
  using G = TmaGeo<NX, TZB>;
  extern __shared__ __align__(1024) float rhs_tma_smem[];
  float* tiles = rhs_tma_smem;                  // [4 slots][NA][AS]
  float* holds = tiles + 4 * (size_t)G::SLOT;   // [4 slots][NH][TZB][NX]
  float* pct = holds + 4 * (size_t)G::HS;       // [jchunk][kPlaneLd]
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(pct + (size_t)kPlaneLd * jchunk);
  const int nz = g.nz, nyc = g.nyc;
  const int tx = threadIdx.x, tz = threadIdx.y;
  const int tid = tz * NX + tx, lane = tid & 31, warp = tid >> 5;
  const int k0 = blockIdx.x * TZB;
  const int jb = blockIdx.y * jchunk, je = min(nyc, jb + jchunk);
  const size_t P = (size_t)nz * NX;

  if (tid == 0) {
    for (int s = 0; s < 4; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fill_plane_table(pct, mt, R, fz, cf.D, jb, je, jchunk, tid, G::NTHR);
  __syncthreads();
  const bool fuse = fz.on != 0;   // uniform per launch
  FwdCarry<float> fd{0.f, 0.f, 0.f, 0.f, 0.f};

  const bool read_h = cf.zet != 0.f, keep_h = cf.keep_h != 0;   // uniform per launch
  // plane q of the window [jb - 1, je] into slot n & 3, n = q - jb + 1 (warp 0)
  auto issue = [&](int q) {
    const int slot = (q - jb + 1) & 3;
    const bool hq = read_h && q >= jb && q < je;
    unsigned bytes = 0;
#pragma unroll
    for (int a = 0; a < NA; ++a)
      if (q >= 0 && q < (a == AV ? nyc + 1 : nyc)) bytes += G::ROWS * NX * sizeof(float);
    if (hq) bytes += G::HS * sizeof(float);
    if (lane == 0) mbar_arrive_expect_tx(&bars[slot], bytes);
    __syncwarp();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    constexpr int NTILE = NA * G::ROWS * G::NBOX;
    const int nall = NTILE + (hq ? NH * TZB * G::NBOX : 0);
    for (int c = lane; c < nall; c += 32) {
      if (c < NTILE) {
        const int a = c / (G::ROWS * G::NBOX), rr = (c / G::NBOX) % G::ROWS, bx = c % G::NBOX;
        if (q < 0 || q >= (a == AV ? nyc + 1 : nyc)) continue;
        float* dst = tiles + ((size_t)slot * NA + a) * G::AS + rr * G::S + 32 + bx * G::BW;
        tma_row(dst, &maps.t[a], bx * G::BW, (k0 - 1 + rr) & (nz - 1), q, &bars[slot]);
      } else {
        const int c2 = c - NTILE;
        const int h = c2 / (TZB * G::NBOX), rr = (c2 / G::NBOX) % TZB, bx = c2 % G::NBOX;
        float* dst = holds + (size_t)slot * G::HS + (h * TZB + rr) * NX + bx * G::BW;
        tma_row(dst, &maps.h[h], bx * G::BW, k0 + rr, q, &bars[slot]);
      }
    }
  };
  // periodic x-halo of every row of plane q's slot, from inside shared memory
  auto halo = [&](int q) {
    float* ts = tiles + (size_t)((q - jb + 1) & 3) * G::SLOT;
    for (int e = tid; e < NA * G::ROWS * 2; e += G::NTHR) {
      float* row = ts + (e / (2 * G::ROWS)) * G::AS + ((e >> 1) % G::ROWS) * G::S;
      if (e & 1) row[32 + NX] = row[32];
      else row[31] = row[32 + NX - 1];
    }
  };
  if (warp == 0)
    for (int q = jb - 1; q <= min(jb + 2, je); ++q) issue(q);
  int issued = min(jb + 2, je);   // last plane issued (uniform across the block)

  const size_t ck = (size_t)(k0 + tz) * NX + tx;
  float ub, ut, wb, wt;
  wall_values(f, P, ck, cf.Uw, ub, ut, wb, wt);
  const CellK<float> kc{ub, ut, wb, wt};
  const int co = (tz + 1) * G::S + 32 + tx;   // this cell in array 0 of a slot
  YCarry<float> cy{0.f, 0.f, 0.f, 0.f, 0.f};
  int waited = jb - 2;   // last plane this thread has seen land
  bool bad = false;
  for (int j = jb; j < je; ++j) {
    for (int q = waited + 1; q <= j + 1; ++q) {
      const int n = q - jb + 1;
      if (!mbar_wait(&bars[n & 3], (n >> 2) & 1)) {
        bad = true;
        break;
      }
      waited = q;
      halo(q);
    }
    if (__syncthreads_or(bad)) {
      bad = true;
      break;
    }
    const int n0 = j - jb + 1;
    const float* bm = tiles + (size_t)((n0 + 3) & 3) * G::SLOT + co;
    const float* bo = tiles + (size_t)(n0 & 3) * G::SLOT + co;
    const float* bp = tiles + (size_t)((n0 + 1) & 3) * G::SLOT + co;
    const float* hs = holds + (size_t)(n0 & 3) * G::HS + tz * NX + tx;
    float Ho[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (read_h) {
#pragma unroll
      for (int h = 0; h < 5; ++h) Ho[h] = hs[h * TZB * NX];
    }
    const PlaneC q = plane_consts(pct + (size_t)(j - jb) * kPlaneLd);
    CellOut<float> o = rhs_cell_at<float, G::AS, G::S>(j, jb, nyc, bm, bo, bp, Ho, q, kc, cf, cy);
    if (fuse) fuse_forward(o, q, j, jb, fd);
    store_cell(f, rcp, rcm, sh, (size_t)j * P + ck, j > 0, keep_h, o);
    __syncthreads();   // slot of plane j - 1 is free
    if (j + 3 <= je) {
      if (warp == 0) issue(j + 3);
      issued = j + 3;
    }
  }
  if (bad) {
    if (tid == 0) {
      atomicExch(err, PNP_ERR_TIMEOUT);
      // let the copies still in flight land before the shared memory is released
      for (int q = jb - 1; q <= issued; ++q) {
        const int n = q - jb + 1;
        mbar_wait(&bars[n & 3], (n >> 2) & 1);
      }
    }
    __syncthreads();
  }
}

// Rows per block of the TMA kernel for this nx (512 threads), 0 when unsupported.
int rhs_tma_rows(int nx) {
  switch (nx) {
    case 32: return 16;
    case 64: return 8;
    case 128: return 4;
    case 256: return 2;
    default: return 0;
  }
}

}  // namespace

cudaError_t launch_wait_selftest(int* err, double limit_s, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(err, (unsigned long long)(limit_s * 1e9));
  return cudaGetLastError();
}

bool rhs_tma_eligible(const Geo& g) {
  const int tzb = rhs_tma_rows(g.nx);
  return tzb > 0 && g.nz % tzb == 0;
}

cudaError_t build_rhs_maps(RhsMaps* m, const Fields<float>& f, const Shadows& sh, const Geo& g) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult qr;
    void* fn = nullptr;
    const cudaError_t e =
        cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
    if (e != cudaSuccess || qr != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const int bw = g.nx < 256 ? g.nx : 256;
  auto make = [&](CUtensorMap* t, const float* p, int planes) {
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.nz, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nx * sizeof(float), (cuuint64_t)g.nx * g.nz * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)bw, 1, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return encode(t, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(p), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  const float* tin[7] = {f.u, f.w, f.v, f.p, sh.phi, sh.cp, sh.cm};
  const float* hin[5] = {f.Hu, f.Hw, f.Hv, sh.Hcp, sh.Hcm};
  for (int a = 0; a < 7; ++a)
    if (!make(&m->t[a], tin[a], a == AV ? g.ny : g.nyc)) return cudaErrorInvalidValue;
  for (int h = 0; h < 5; ++h)
    if (!make(&m->h[h], hin[h], h == 2 ? g.ny : g.nyc)) return cudaErrorInvalidValue;
  return cudaSuccess;
}

namespace {
int sm_count() {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      nsm = 152;
  }
  return nsm;
}

// The stencil kernel a launch takes and its y-chunk length.
struct RhsPlan {
  int kind;   // 0: TMA rows; 1: 64-wide pair tile; 2: 32-wide pair tile; 3: one-cell 32 x 8; 4: 8 x 4; 5: 4 x 4
  int tzb;    // TMA: rows per block
  int jc;     // planes per y-chunk
};

// y-chunk length: the best product of wave efficiency (blocks over the
// resident slots, rounded up to whole waves) and chunk efficiency (each chunk
// also loads the planes below and above it), chunks of >= 8 planes
int chunk_len(const Geo& g, int nxz, int per_sm) {
  const int slots = sm_count() * per_sm;
  int best = g.nyc;
  double best_eff = -1.0;
  for (int nch = 1; nch <= (g.nyc + 7) / 8; ++nch) {
    const int jc = (g.nyc + nch - 1) / nch;
    const double blocks = (double)nxz * ((g.nyc + jc - 1) / jc);
    const double waves = blocks / slots;
    const double eff = waves / std::ceil(waves) * jc / (jc + 2.0);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = jc;
    }
  }
  return best;
}

// TMA rows: lc_rhs_bx 128 (when the tensor maps exist); cp.async tiles: the
// default and 64 / 32 / 16.  lc_rhs_bx: 64 = 64 x 4 threads with a packed pair
// of cells each in z (a 64 x 8 tile), old H by direct loads; 32 = the same on
// 32 x 8 threads (a 32 x 16 tile); 0 = the 64-wide tile where nx >= 64, else
// the 32-wide one; 16 = 32 x 8 threads with one cell each, old H on the
// cp.async ring; narrower grids fall back to 8 x 4 / 4 x 4.  Measured on the
// 256x193x256 workload: 0.210 ms (64 wide), 0.224 ms (32 wide), 0.259 ms (one
// cell); 64 x 8 threads (one 512-thread block per SM) 0.220 ms, 128 x 2 0.221 ms
RhsPlan plan_for(const Geo& g, bool tma_maps) {
  const int code = g.lc_rhs_bx;
  if (tma_maps && code == 128 && rhs_tma_eligible(g)) {
    const int tzb = rhs_tma_rows(g.nx);
    return {0, tzb, chunk_len(g, g.nz / tzb, 1)};
  }
  auto tile = [&](int kind, int bx, int bz, int cz, int per_sm) {
    return RhsPlan{kind, 0, chunk_len(g, (g.nx / bx) * (g.nz / (bz * cz)), per_sm)};
  };
  if (g.nx >= 64 && g.nz >= 8 && (code == 64 || code == 0 || code == 128)) return tile(1, 64, 4, 2, 2);
  if (g.nx >= 32 && g.nz >= 16 && code != 16) return tile(2, 32, 8, 2, 2);
  if (g.nx >= 32 && g.nz >= 8) return tile(3, 32, 8, 1, 3);
  if (g.nx >= 8) return tile(4, 8, 4, 1, 24);
  return tile(5, 4, 4, 1, 48);
}
}  // namespace

int mixed_rhs_chunk(const Geo& g, bool tma_maps) { return plan_for(g, tma_maps).jc; }

cudaError_t launch_mixed_rhs(const Fields<float>& f, const Shadows& sh, const MixedRefs& R, const Geo& g,
                             const MetricsF& m, const CoefF& cf, const RhsMaps* maps, int* err, cudaStream_t s,
                             const CnFuse* fuse) {
  float* rp = reinterpret_cast<float*>(f.rcp);
  float* rm = reinterpret_cast<float*>(f.rcm);
  const CnFuse fz = fuse ? *fuse : CnFuse{};
  const RhsPlan pl = plan_for(g, maps != nullptr);
  if (fz.on && fz.jc != pl.jc) return cudaErrorInvalidValue;   // the back substitution's chunks must match
  const int jc = pl.jc;
  if (pl.kind == 0) {
    auto go = [&](auto kern, auto geo, int tzb) {
      using G = decltype(geo);
      const size_t smem = G::bytes(jc);
      if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      const dim3 grd((unsigned)(g.nz / tzb), (unsigned)((g.nyc + jc - 1) / jc));
      kern<<<grd, dim3(g.nx, tzb), smem, s>>>(*maps, f, rp, rm, sh, R, g, m, cf, jc, err, fz);
      return cudaGetLastError();
    };
    switch (g.nx) {
      case 32: return go(k_rhs_mixed_tma<32, 16>, TmaGeo<32, 16>{}, 16);
      case 64: return go(k_rhs_mixed_tma<64, 8>, TmaGeo<64, 8>{}, 8);
      case 128: return go(k_rhs_mixed_tma<128, 4>, TmaGeo<128, 4>{}, 4);
      default: return go(k_rhs_mixed_tma<256, 2>, TmaGeo<256, 2>{}, 2);
    }
  }
  auto go = [&](auto kern, int bx, int bz, int cz, bool hsm) {
    const dim3 grd((unsigned)(g.nx / bx), (unsigned)(g.nz / (bz * cz)), (unsigned)((g.nyc + jc - 1) / jc));
    const size_t smem = sizeof(float) * (rhs_tile_floats(bx, bz, cz, hsm) + (size_t)kPlaneLd * jc);
    if (smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    kern<<<grd, dim3(bx, bz), smem, s>>>(f, rp, rm, sh, R, g, m, cf, jc, fz);
    return cudaGetLastError();
  };
  switch (pl.kind) {
    case 1: return go(k_rhs_mixed_tile<64, 4, 2, false, 2>, 64, 4, 2, false);
    case 2: return go(k_rhs_mixed_tile<32, 8, 2, false, 2>, 32, 8, 2, false);
    case 3: return go(k_rhs_mixed_tile<32, 8, 1, true, 3>, 32, 8, 1, true);
    case 4: return go(k_rhs_mixed_tile<8, 4, 1, true, 24>, 8, 4, 1, true);
    default: return go(k_rhs_mixed_tile<4, 4, 1, true, 32>, 4, 4, 1, true);
  }
}

}  // namespace pnp
