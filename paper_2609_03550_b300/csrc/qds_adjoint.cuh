// qds_adjoint.cuh -- the transpose of one QDS EM + axion step.
//
// For a real functional L of the complex state, the adjoint of a complex
// value z is zb = dL/dRe z + i dL/dIm z; a term y = c x (c complex) gives
// xb += conj(c) yb, and y = conj(x) gives xb += conj(yb).  The regenerated
// group never feeds back into the EM fields or the axion (Sec. 2.2, reading
// of the step order), so the adjoint of an axion-energy functional has no
// regenerated part and this transpose covers the EM group and the axion.
//
// Adjoint fields live in the canonical window-order layout (no ring offset)
// in the working precision.  The forward state of the step (time n) is read
// through a Tile with s = 0 (its window order).  The step is transposed pass
// by pass in reverse order of the forward passes:
//   AD_UNPHI   window shift and phi update (Eq. phi_update)
//   AD_UNTA    T_a shift (Eqs. Ta_plus_update, Ta_minus_update)
//   AD_UNSHIFT T shift, its face sources and the outer box (Eqs. Trp/Trm/
//              Ttp/Ttm_update, axis_Ttheta, em_r_open_bt)
//   AD_UNSRC   Gamma_a: Laplacian, mass, the outer ghost and the bilinear
//              source S_a (Eq. mode_convolution), d L / d g accumulated
//   AD_UNLEAP  E_x, B_x leapfrog and the outer box (Eqs. Ex_update,
//              axis_Ex, em_r_open_bx)
// The transpose of the +x shift is the -x shift and vice versa.  Open x,
// open r, optional moving window; no periodic or closed test modes.
#pragma once

#include "qds_stages.cuh"

namespace qds {

enum AdStage { AD_UNPHI = 0, AD_UNTA, AD_UNSHIFT, AD_UNSRC, AD_UNLEAP, N_ADSTAGE };

// scratch planes of the adjoint (window order), each M*nx*nr
enum AdScr { SB_TRP = 0, SB_TRM, SB_TTP, SB_TTM, SB_EX, SB_BX, SB_TAP, SB_TAM, SB_G, N_SB };

template <class R>
QDS_HD void cadd(C<R> *p, C<R> v) {
#if defined(__CUDA_ARCH__)
  atomicAdd(&p->re, v.re);
  atomicAdd(&p->im, v.im);
#else
  p->re += v.re;
  p->im += v.im;
#endif
}

template <class R, int M>
struct Adj {
  Tile<R, M, false> f;  // forward state at time n (s = 0)
  const C<R> *ln;              // adjoint of the state after the step
  C<R> *lo;                    // adjoint of the state before the step (accumulated)
  C<R> *sb;                    // scratch planes
  double *dg;                  // accumulated dL/dg (null: not wanted)
  int nx, nr, J;
  size_t P;
  bool mw;
  R h, dr, ih, idr;
  R gs, ma2;

  QDS_HD size_t ai(int field, int k, int w, int j) const { return ((size_t)field * M + k) * (size_t)nx * nr + (size_t)w * nr + j; }
  QDS_HD bool in_cell(int w) const { return w >= 0 && w < nx; }
  QDS_HD bool in_face(int w) const { return w >= 0 && w <= nx - 2; }
  // adjoint of the new state in the fixed box (before the window shift)
  QDS_HD C<R> lnew(int field, int k, int w, int j) const {
    if (mw) w -= 1;
    if (w < 0 || w >= nx || j < 0 || j >= nr) return zero<R>();
    return ln[ai(field, k, w, j)];
  }
  QDS_HD C<R> lnew_prev(int k, int w) const {
    if (mw) w -= 1;
    if (w < 0 || w >= nx) return zero<R>();
    return ln[(size_t)NFIELD * P + (size_t)k * nx + w];
  }
  QDS_HD C<R> &old(int field, int k, int w, int j) const { return lo[ai(field, k, w, j)]; }
  QDS_HD C<R> *oldp(int field, int k, int w, int j) const { return lo + ai(field, k, w, j); }
  QDS_HD C<R> *oldprev(int k, int w) const { return lo + (size_t)NFIELD * P + (size_t)k * nx + w; }
  QDS_HD C<R> &s(int plane, int k, int w, int j) const { return sb[((size_t)plane * M + k) * (size_t)nx * nr + (size_t)w * nr + j]; }
  QDS_HD C<R> sv(int plane, int k, int w, int j) const {
    if (w < 0 || w >= nx || j < 0 || j >= nr) return zero<R>();
    return s(plane, k, w, j);
  }
  // scatter into the old adjoint of a transverse field at a cell (E_r, B_th,
  // E_th, B_r -> T^+-), ignoring positions outside the box
  QDS_HD void add_Er(int k, int c, int j, C<R> v) const { if (in_cell(c)) { cadd(oldp(TRP, k, c, j), R(0.5) * v); cadd(oldp(TRM, k, c, j), R(0.5) * v); } }
  QDS_HD void add_Bt(int k, int c, int j, C<R> v) const { if (in_cell(c)) { cadd(oldp(TRP, k, c, j), R(0.5) * v); cadd(oldp(TRM, k, c, j), R(-0.5) * v); } }
  QDS_HD void add_Et(int k, int c, int j, C<R> v) const { if (in_cell(c)) { cadd(oldp(TTP, k, c, j), R(0.5) * v); cadd(oldp(TTM, k, c, j), R(0.5) * v); } }
  QDS_HD void add_Br(int k, int c, int j, C<R> v) const { if (in_cell(c)) { cadd(oldp(TTP, k, c, j), R(0.5) * v); cadd(oldp(TTM, k, c, j), R(-0.5) * v); } }
};

// Transpose of the mode convolution C_m{A, B} (Eq. mode_convolution) for all
// output modes at once: Ab += dC/dA^T Sb, Bb += dC/dB^T Sb (scaled by wgt).
template <class R, int M>
QDS_HD void conv_T(const C<R> *A, const C<R> *B, const C<R> *Sb, R wgt, C<R> *Ab, C<R> *Bb) {
  // m = 0: A0 B0 + (1/2) sum_k Re(A_k conj B_k)
  {
    C<R> s0 = wgt * Sb[0];
    Ab[0] += mul_cj(s0, B[0]);
    Bb[0] += mul_cj(s0, A[0]);
    for (int k = 1; k < M; k++) {
      Ab[k] += (R(0.5) * s0.re) * B[k];
      Bb[k] += (R(0.5) * s0.re) * A[k];
    }
  }
  for (int m = 1; m < M; m++) {
    C<R> t = (R(0.5) * wgt) * Sb[m];
    for (int k = 0; k <= m && k < M; k++) {  // A_k B_l, k + l = m
      int l = m - k;
      if (l < M) {
        Ab[k] += mul_cj(t, B[l]);
        Bb[l] += mul_cj(t, A[k]);
      }
    }
    for (int l = 0; l + m < M; l++) {  // A_{l+m} conj(B_l)
      Ab[l + m] += B[l] * t;
      Bb[l] += mul_cj(A[l + m], t);
    }
    for (int k = 0; k + m < M; k++) {  // conj(A_k) B_{k+m}
      Ab[k] += mul_cj(B[k + m], t);
      Bb[k + m] += A[k] * t;
    }
  }
}

// ---------------------------------------------------------------------------
template <class R, int M>
QDS_HD void adj_point(const Adj<R, M> &a, int st, int w, int j, double &dg_acc) {
  const int J = a.J;
  const R h = a.h, dr = a.dr, idr = a.idr;
  const R ka = R(0.5) * a.ih, kb = R(0.5) * idr;  // box-scheme weights
  const Tile<R, M, false> &t = a.f;

  if (st == AD_UNPHI) {
    // phi^(n+1) = phi^n + (h/4) sum T_a^(n+1/2) over the cells around face w;
    // phi_prev^(n+1) = phi^n on the last row.  Also seeds the scratch with
    // the adjoints of the new T, E_x, B_x (window shift undone).
    for (int k = 0; k < M; k++) {
      for (int q = 0; q < 4; q++) a.s(SB_TRP + q, k, w, j) = a.lnew(TRP + q, k, w, j);
      a.s(SB_EX, k, w, j) = a.in_face(w) ? a.lnew(EX, k, w, j) : zero<R>();
      a.s(SB_BX, k, w, j) = a.in_face(w) ? a.lnew(BX, k, w, j) : zero<R>();
      C<R> pl = a.in_face(w - 1) ? a.lnew(PHI, k, w - 1, j) : zero<R>();
      C<R> pr = a.in_face(w) ? a.lnew(PHI, k, w, j) : zero<R>();
      C<R> tp = a.lnew(TAP, k, w, j) + (R(0.25) * h) * (pl + pr);
      C<R> tm = a.lnew(TAM, k, w, j) + (R(0.25) * h) * (pl + pr);
      a.s(SB_TAP, k, w, j) = tp;
      a.s(SB_TAM, k, w, j) = tm;
      C<R> ph = pr;
      if (j == J && a.in_face(w)) ph += a.lnew_prev(k, w);
      a.old(PHI, k, w, j) = ph;
      if (j == 0) *a.oldprev(k, w) = zero<R>();
      // scatter targets start at zero; the regenerated group has no adjoint
      for (int fl = TRP; fl <= BX; fl++) a.old(fl, k, w, j) = zero<R>();
      for (int fl = TRP1; fl < NFIELD; fl++) a.old(fl, k, w, j) = zero<R>();
    }
    return;
  }
  if (st == AD_UNTA) {
    // T_a^+(c) = T_a^+(c-1) + h G(c-1);  T_a^-(c) = T_a^-(c+1) + h G(c)
    for (int k = 0; k < M; k++) {
      a.s(SB_G, k, w, j) = a.in_face(w) ? h * (a.sv(SB_TAP, k, w + 1, j) + a.sv(SB_TAM, k, w, j)) : zero<R>();
      a.old(TAP, k, w, j) = a.sv(SB_TAP, k, w + 1, j);
      a.old(TAM, k, w, j) = a.sv(SB_TAM, k, w - 1, j);
    }
    return;
  }
  if (st == AD_UNSHIFT) {
    for (int k = 0; k < M; k++) {
      // adjoints of the new T at cell c (effective: with the fold of the
      // outer box into row J-1 for T_r)
      auto boxBt = [&](int c) -> C<R> {  // adjoint of B_th^(n+1) on the last half row at cell c
        return a.sv(SB_TRP, k, c, J) - a.sv(SB_TRM, k, c, J);
      };
      auto trpn = [&](int c, int jj) -> C<R> {
        if (!a.in_cell(c)) return zero<R>();
        C<R> v = a.s(SB_TRP, k, c, jj);
        if (jj == J - 1) v += (R(0.5) * (-(ka - kb) / (ka + kb))) * boxBt(c);
        return v;
      };
      auto trmn = [&](int c, int jj) -> C<R> {
        if (!a.in_cell(c)) return zero<R>();
        C<R> v = a.s(SB_TRM, k, c, jj);
        if (jj == J - 1) v -= (R(0.5) * (-(ka - kb) / (ka + kb))) * boxBt(c);
        return v;
      };
      auto ttn = [&](int plane, int c, int jj) -> C<R> {
        if (!a.in_cell(c)) return zero<R>();
        if (jj == 0 && k != 1) return zero<R>();
        return a.s(plane, k, c, jj);
      };
      // ---- the old T at cell w: the shifted copies (-x for T_r^+, T_th^-,
      // +x for T_r^-, T_th^+) ----
      {
        const int c = w;
        if (j < J) {
          cadd(a.oldp(TRP, k, c, j), trpn(c + 1, j));
          cadd(a.oldp(TRM, k, c, j), trmn(c - 1, j));
        } else {
          // last half row: E_r^(n+1)(c') = (T_r^+(c'-1) + T_r^-(c'+1))/2 + ...
          C<R> er_r = a.sv(SB_TRP, k, c + 1, J) + a.sv(SB_TRM, k, c + 1, J);
          C<R> er_l = a.sv(SB_TRP, k, c - 1, J) + a.sv(SB_TRM, k, c - 1, J);
          if (a.in_cell(c + 1)) cadd(a.oldp(TRP, k, c, J), R(0.5) * er_r);
          if (a.in_cell(c - 1)) cadd(a.oldp(TRM, k, c, J), R(0.5) * er_l);
        }
        cadd(a.oldp(TTP, k, c, j), ttn(SB_TTP, c - 1, j));
        cadd(a.oldp(TTM, k, c, j), ttn(SB_TTM, c + 1, j));
      }
      // ---- the outer T_r box of cell w (last half row): old-field terms ----
      if (j == J) {
        const int c = w;
        const R rJ = R(J) * dr;
        C<R> Bb = boxBt(c);
        if (Bb.re != R(0) || Bb.im != R(0)) {
          // B_th^(n+1) = (R - (a-b) bt_in_new + (a-b) Bo + (a+b) Bi)/(a+b)
          a.add_Bt(k, c, J, ((ka - kb) / (ka + kb)) * Bb);
          a.add_Bt(k, c, J - 1, Bb);
          C<R> Rb = (R(1) / (ka + kb)) * Bb;
          // R = -(1/4)(ih)(Er_r - Er_l) - (1/2 rJ)(Bth + i k Br) + (1/4)(jx..)
          C<R> er = (R(-0.125) * t.ih) * Rb;
          a.add_Er(k, c + 1, J - 1, er);
          a.add_Er(k, c + 1, J, er);
          a.add_Er(k, c - 1, J - 1, -er);
          a.add_Er(k, c - 1, J, -er);
          a.add_Bt(k, c, J - 1, (R(-0.25) / rJ) * Rb);
          a.add_Bt(k, c, J, (R(-0.25) / rJ) * Rb);
          a.add_Br(k, c, J, imul(R(k) * R(0.5) / rJ, Rb));  // conj(-i k/(2 rJ)) = i k/(2 rJ)
        }
      }
      // ---- face w: adjoints of the sources, gathered into E_x, B_x ----
      if (a.in_face(w)) {
        const int f = w;
        // source adjoints at face f, row jj
        auto Sr = [&](int jj, C<R> &Gb, C<R> &Pb) {  // T_r sources (half row jj < J)
          C<R> sp = h * trpn(f + 1, jj), sm = h * trmn(f, jj);
          Gb = sp + sm;
          Pb = sp - sm;
        };
        auto St = [&](int jj, C<R> &Gb, C<R> &Pb) {  // T_th sources (row jj)
          C<R> sp = h * ttn(SB_TTP, f, jj), sm = h * ttn(SB_TTM, f + 1, jj);
          Gb = sp + sm;
          Pb = sp - sm;
        };
        C<R> ex = zero<R>(), bx = zero<R>();
        C<R> Gr, Pr, Gt, Pt;
        // E_x^(n+1/2)(f, j): Phi_r(f, j) = (Ex(j+1) - Ex(j))/dr, Phi_r(f, j-1), Phi_th
        if (j < J) { Sr(j, Gr, Pr); ex -= idr * Pr; }
        if (j >= 1 && j - 1 < J) { Sr(j - 1, Gr, Pr); ex += idr * Pr; }
        if (j >= 1) { St(j, Gt, Pt); ex += imul(-R(k) / (R(j) * dr), Pt); }
        if (k == 1 && j <= 1) {  // axis Phi_th = i (Ex(1) - Ex(0))/dr
          St(0, Gt, Pt);
          ex += imul(j == 1 ? -idr : idr, Pt);
        }
        // B_x^(n+1/2)(f, j): Gamma_r(f, j), Gamma_th(f, j), Gamma_th(f, j+1)
        const R rh = (R(j) + R(0.5)) * dr;
        if (j < J) { Sr(j, Gr, Pr); bx += imul(R(k) / rh, Gr); }
        else {
          // E_r^(n+1) on the last row takes Gamma_r of faces c-1 and c:
          C<R> Gb = (R(0.5) * h) * (a.sv(SB_TRP, k, f + 1, J) + a.sv(SB_TRM, k, f + 1, J) +
                                     a.sv(SB_TRP, k, f, J) + a.sv(SB_TRM, k, f, J));
          bx += imul(R(k) / rh, Gb);
        }
        if (j >= 1) { St(j, Gt, Pt); bx -= idr * Gt; }
        else if (k == 1) { St(0, Gt, Pt); bx += (-R(2) * idr) * Gt; }
        if (j + 1 <= J && j + 1 >= 1) { St(j + 1, Gt, Pt); bx += idr * Gt; }
        a.s(SB_EX, k, f, j) += ex;
        a.s(SB_BX, k, f, j) += bx;
      }
    }
    return;
  }
  if (st == AD_UNSRC) {
    if (!a.in_face(w)) return;
    const int f = w;
    const bool top = (j == J);
    const R rh = (R(j) + R(0.5)) * dr;
    const R den = R(1) / ((R(j) + R(0.5)) * dr * dr);
    // phi adjoint from Gamma_a of rows j-1, j, j+1 (Laplacian and mass)
    C<R> Gb[M];
    for (int k = 0; k < M; k++) {
      Gb[k] = a.s(SB_G, k, f, j);
      C<R> v = zero<R>();
      // row j itself
      {
        R cc = -(R(2 * j + 1)) * den - (R(k * k) / (rh * rh) + a.ma2);
        if (top) cc += R(J + 1) * den * (-R(2) * dr * t.ih);  // ghost: -(2 dr/h) phi(J)
        v += cc * Gb[k];
      }
      if (j >= 1) {  // row j-1 uses phi(j) as its upper neighbour
        const int i = j - 1;
        const R di = R(1) / ((R(i) + R(0.5)) * dr * dr);
        v += (R(i + 1) * di) * a.s(SB_G, k, f, i);
      }
      if (j + 1 <= J) {  // row j+1 uses phi(j) as its lower neighbour
        const int i = j + 1;
        const R di = R(1) / ((R(i) + R(0.5)) * dr * dr);
        C<R> g1 = a.s(SB_G, k, f, i);
        v += (R(i) * di) * g1;
        if (i == J) v += (R(J + 1) * di) * g1;  // ghost of row J: + phi(J-1)
      }
      cadd(a.oldp(PHI, k, f, j), v);
      if (top) cadd(a.oldprev(k, f), (R(J + 1) * den * R(2) * dr * t.ih) * Gb[k]);
    }
    // source: Gamma_a += gs S;  S = C{eX, bX} + (1/2)(C{rp, qp} - C{rm, qm})
    C<R> Sb[M];
    for (int m = 0; m < M; m++) Sb[m] = a.gs * Gb[m];
    C<R> eX[M], bX[M], rp[M], rm[M], qp[M], qm[M];
    C<R> exn[M], exn1[M], bxn[M];
    for (int k = 0; k < M; k++) {
      exn[k] = ex_update(t, 0, k, f, j, t.srcv(t.jx, k, f, j));
      bxn[k] = (j < J) ? bx_interior(t, 0, k, f, j)
                       : bx_outer(t, 0, k, f, R(0.5) * (t.srcv(t.jt, k, f, j) + t.srcv(t.jt, k, f + 1, j)),
                                  bx_interior(t, 0, k, f, j - 1));
      exn1[k] = top ? exn[k] : ex_update(t, 0, k, f, j + 1, t.srcv(t.jx, k, f, j + 1));
      C<R> eo = t.face(EX, k, f, j), eo1 = top ? eo : t.face(EX, k, f, j + 1);
      eX[k] = R(0.25) * (eo + eo1 + exn[k] + exn1[k]);
      bX[k] = R(0.5) * (t.face(BX, k, f, j) + bxn[k]);
      const int j1 = top ? j : j + 1;
      rp[k] = R(0.5) * (t.cell(TRP, k, f, j) + t.cell(TRP, k, f + 1, j));
      rm[k] = R(0.5) * (t.cell(TRM, k, f, j) + t.cell(TRM, k, f + 1, j));
      qp[k] = R(0.25) * (t.cell(TTP, k, f, j) + t.cell(TTP, k, f + 1, j) + t.cell(TTP, k, f, j1) + t.cell(TTP, k, f + 1, j1));
      qm[k] = R(0.25) * (t.cell(TTM, k, f, j) + t.cell(TTM, k, f + 1, j) + t.cell(TTM, k, f, j1) + t.cell(TTM, k, f + 1, j1));
    }
    if (a.dg) {  // dL/dg: Gamma_a depends on g through g S (physical variables)
      double acc = 0;
      for (int m = 0; m < M; m++) {
        C<R> S = conv<R, M>(m, eX, bX) + R(0.5) * (conv<R, M>(m, rp, qp) - conv<R, M>(m, rm, qm));
        S += t.srcv(t.sext, m, f, j);
        acc += (double)Gb[m].re * S.re + (double)Gb[m].im * S.im;
      }
      dg_acc += acc;  // the caller reduces and adds to *a.dg
    }
    C<R> eXb[M], bXb[M], rpb[M], rmb[M], qpb[M], qmb[M];
    for (int k = 0; k < M; k++) eXb[k] = bXb[k] = rpb[k] = rmb[k] = qpb[k] = qmb[k] = zero<R>();
    conv_T<R, M>(eX, bX, Sb, R(1), eXb, bXb);
    conv_T<R, M>(rp, qp, Sb, R(0.5), rpb, qpb);
    conv_T<R, M>(rm, qm, Sb, R(-0.5), rmb, qmb);
    for (int k = 0; k < M; k++) {
      // eX = (Ex(j) + Ex(j1) + Exn(j) + Exn(j1))/4, j1 = j on the last row
      C<R> e4 = R(0.25) * eXb[k];
      cadd(a.oldp(EX, k, f, j), e4);
      cadd(&a.s(SB_EX, k, f, j), e4);
      const int j1 = top ? j : j + 1;
      cadd(a.oldp(EX, k, f, j1), e4);
      cadd(&a.s(SB_EX, k, f, j1), e4);
      cadd(a.oldp(BX, k, f, j), R(0.5) * bXb[k]);
      cadd(&a.s(SB_BX, k, f, j), R(0.5) * bXb[k]);
      for (int dc = 0; dc < 2; dc++) {
        if (!a.in_cell(f + dc)) continue;
        cadd(a.oldp(TRP, k, f + dc, j), R(0.5) * rpb[k]);
        cadd(a.oldp(TRM, k, f + dc, j), R(0.5) * rmb[k]);
        cadd(a.oldp(TTP, k, f + dc, j), R(0.25) * qpb[k]);
        cadd(a.oldp(TTM, k, f + dc, j), R(0.25) * qmb[k]);
        cadd(a.oldp(TTP, k, f + dc, j1), R(0.25) * qpb[k]);
        cadd(a.oldp(TTM, k, f + dc, j1), R(0.25) * qmb[k]);
      }
    }
    return;
  }
  if (st == AD_UNLEAP) {
    if (!a.in_face(w)) return;
    const int f = w;
    for (int k = 0; k < M; k++) {
      // ---- E_x^(n+1/2) = E_x^(n-1/2) + h Gamma_x (Eqs. Ex_update, axis_Ex) ----
      const C<R> eb = a.s(SB_EX, k, f, j);
      if (j == 0) {
        if (k == 0) {  // h (4/dr) (Bt(f,0) + Bt(f+1,0))/2
          cadd(a.oldp(EX, k, f, 0), eb);
          C<R> v = (h * R(2) * idr) * eb;
          a.add_Bt(k, f, 0, v);
          a.add_Bt(k, f + 1, 0, v);
        }  // m != 0: E_x is held at zero on the axis
      } else {
        cadd(a.oldp(EX, k, f, j), eb);
        const R rj = R(j) * dr;
        C<R> bhi = (h * (R(j) + R(0.5)) / rj) * eb, blo = (-h * (R(j) - R(0.5)) / rj) * eb;
        C<R> brb = imul(-h * R(k) / rj, eb);  // conj(h i k / r_j)
        for (int dc = 0; dc < 2; dc++) {
          a.add_Bt(k, f + dc, j, R(0.5) * bhi);
          a.add_Bt(k, f + dc, j - 1, R(0.5) * blo);
          a.add_Br(k, f + dc, j, R(0.5) * brb);
        }
      }
      // ---- B_x^(n+1/2) (Eq. Phix_explicit; outer row: Eq. em_r_open_bx) ----
      C<R> bbar = a.s(SB_BX, k, f, j);
      if (j == J - 1) bbar += (-(ka - kb) / (ka + kb)) * a.s(SB_BX, k, f, J);  // box uses B_x^(n+1/2)(J-1)
      if (j < J) {
        cadd(a.oldp(BX, k, f, j), bbar);
        const R rh = (R(j) + R(0.5)) * dr;
        C<R> ehi = (-h * R(j + 1) / rh) * bbar, elo = (h * R(j) / rh) * bbar;
        C<R> erb = imul(h * R(k) / rh, bbar);  // conj(-h i k / r_{j+1/2})
        for (int dc = 0; dc < 2; dc++) {
          a.add_Et(k, f + dc, j + 1, R(0.5) * ehi);
          a.add_Et(k, f + dc, j, R(0.5) * elo);
          a.add_Er(k, f + dc, j, R(0.5) * erb);
        }
      } else {
        // B_x(J) = (R - (a-b) B_x^(n+1/2)(J-1) + (a-b) B_x(J) + (a+b) B_x(J-1))/(a+b)
        cadd(a.oldp(BX, k, f, J), ((ka - kb) / (ka + kb)) * bbar);
        cadd(a.oldp(BX, k, f, J - 1), bbar);
        const C<R> Rb = (R(1) / (ka + kb)) * bbar;
        const R rJ = R(J) * dr;
        // R = (1/2) ih (Br(f+1,J) - Br(f,J)) - (1/(2 rJ)) (Eth + i k Er4) - jt/2
        a.add_Br(k, f + 1, J, (R(0.5) * t.ih) * Rb);
        a.add_Br(k, f, J, (R(-0.5) * t.ih) * Rb);
        a.add_Et(k, f, J, (R(-0.25) / rJ) * Rb);
        a.add_Et(k, f + 1, J, (R(-0.25) / rJ) * Rb);
        C<R> er4 = imul(R(k) * R(0.125) / rJ, Rb);  // (1/4) conj(-i k/(2 rJ))
        a.add_Er(k, f, J - 1, er4);
        a.add_Er(k, f, J, er4);
        a.add_Er(k, f + 1, J - 1, er4);
        a.add_Er(k, f + 1, J, er4);
      }
    }
    return;
  }
}

}  // namespace qds
