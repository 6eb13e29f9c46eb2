#include <algorithm>
// qds_emu.cpp -- host emulation of the fused step kernel, for CPU tests only.
//
// Compiles the same stage code as the CUDA kernel (qds_stages.cuh) for the
// host with bounds checks on every global and shared-memory access, and runs
// each tile's stages in kernel order (all threads of a stage before the next
// stage).  It exists so that the tile indexing can be checked on the CPU
// before the kernel runs on a GPU; it is a separate library (libqds_emu.so)
// that the product path never loads.
#define QDS_EMU 1
#include <cstring>
#include <vector>

#include "qds_stages.cuh"

using namespace qds;

namespace {

template <class R, int M>
void emu_steps(const double *canon, double *out, int nx, int nr, double h, double dr, double m_a, double g,
               uint32_t flags, const double *jx, const double *jr, const double *jt, const double *sext,
               int nsteps, int TX, int TR, int nthreads, int fused) {
  const size_t P = plane_elems(M, nx, nr), E = state_elems(M, nx, nr);
  const bool sc = (flags & (F_FP32 | F_SCALE_G)) && g != 0.0;
  const double s_ax = sc ? 1.0 / g : 1.0, s_ar = sc ? 1.0 / (g * g) : 1.0;
  std::vector<C<R>> buf[2];
  buf[0].resize(E);
  buf[1].resize(E);
  for (size_t q = 0; q < E; q++) {
    double sc_ = 1.0;
    if (q < (size_t)NFIELD * P) {
      int f = (int)(q / P);
      if (f == PHI || f == TAP || f == TAM) sc_ = s_ax;
      else if (f >= TRP1) sc_ = s_ar;
    } else sc_ = s_ax;
    buf[0][q] = buf[1][q] = mk<R>((R)(canon[2 * q] * sc_), (R)(canon[2 * q + 1] * sc_));
  }
  std::vector<C<R>> sj[4];
  const double *srcs[4] = {jx, jr, jt, sext};
  for (int a = 0; a < 4; a++)
    if (srcs[a]) {
      sj[a].resize(P);
      for (size_t q = 0; q < P; q++) sj[a][q] = mk<R>((R)srcs[a][2 * q], (R)srcs[a][2 * q + 1]);
    }
  Inst<R> I;
  std::memset(&I, 0, sizeof I);
  I.nx = nx; I.nr = nr; I.M = M; I.flags = flags;
  I.h = (R)h; I.dr = (R)dr; I.inv_h = (R)(1.0 / h); I.inv_dr = (R)(1.0 / dr);
  I.ma2 = (R)(m_a * m_a);
  I.gs = sc ? (R)1 : (R)g;
  I.gj = sc ? (R)1 : (R)g;
  I.jx = jx ? sj[0].data() : nullptr;
  I.jr = jr ? sj[1].data() : nullptr;
  I.jt = jt ? sj[2].data() : nullptr;
  I.sext = sext ? sj[3].data() : nullptr;
  Geo geo;
  geo.TX = TX;
  geo.TR = TR;
  Smem L = smem_layout(geo, M, flags);
  std::vector<C<R>> sm(L.total);
  std::vector<C<R>> scratch(4 * P);
  for (int q = 0; q < (int)scratch.size(); q++) scratch[q] = mk<R>((R)1e30, (R)1e30);
  I.scratch = scratch.data();
  auto pass_tile_at = [&](int n, int x0, int r0) {
    Tile<R, M, false, false> t;
    t.bind(I, &I);
    t.nx = nx; t.nr = nr; t.J = nr - 1;
    t.x0 = x0; t.r0 = r0;
    t.per = (flags & F_X_PERIODIC) != 0;
    t.closed = (flags & F_R_CLOSED) != 0;
    t.mw = (flags & F_MOVING_WINDOW) != 0;
    t.s = t.mw ? n % nx : 0;
    t.P = P;
    t.o = buf[n & 1].data();
    t.n = buf[(n & 1) ^ 1].data();
    t.h = I.h; t.dr = I.dr; t.ih = I.inv_h; t.idr = I.inv_dr;
    t.g = Geo{};
    t.g.TX = 8; t.g.TR = 32;
    t.L = Smem{};
    t.sm = nullptr;
    t.scr = scratch.data();
    t.state_len = E;
    t.sm_len = 0;
    return t;
  };
  // pass mode (fused == 0): the warp-column passes P1, P2, then the
  // regenerated shift and the window zeroing as stage passes; warps and
  // lanes run in order, phase 1 of all 32 lanes before phase 2
  for (int n = 0; n < nsteps && fused == 0; n++) {
    const bool ar = (flags & F_AREM) != 0, mw = (flags & F_MOVING_WINDOW) != 0;
    const bool per_ = (flags & F_X_PERIODIC) != 0;
    for (int pass = 1; pass <= 2; pass++) {
      const int stride = pass == 1 ? 31 : 30;
      for (int x0 = 0; x0 < nx; x0 += 8)
        for (int r0 = 0; r0 < nr; r0 += stride) {
          const bool inner = per_ ? (nx >= 8 + 4) : (x0 >= 2 && x0 + 8 + 2 <= nx - 1);
          const int base = pass == 1 ? r0 : (r0 > 0 ? r0 - 1 : 0);
          Tile<R, M, false, false> t = pass_tile_at(n, x0, base);
          Tile<R, M, false, true> tf;
          std::memcpy((void *)&tf, (const void *)&t, sizeof t);
          for (int lx = 0; lx < 8 && x0 + lx < nx; lx++) {
            std::vector<P1Lane<R, M>> L1(32);
            std::vector<P2Lane<R, M>> L2(32);
            for (int ph = 0; ph < 2; ph++)
              for (int lane = 0; lane < 32; lane++) {
                const int j = base + lane;
                const bool out = pass == 1 ? (lane < 31 && j < nr) : (j >= r0 && j < r0 + 30 && j < nr);
                if (pass == 1 && ph == 0) { if (inner) p1_leap(tf, lx, lane, out, L1[lane]); else p1_leap(t, lx, lane, out, L1[lane]); }
                if (pass == 1 && ph == 1) { if (inner) p1_source(tf, lx, lane, out, L1.data()); else p1_source(t, lx, lane, out, L1.data()); }
                if (pass == 2 && ph == 0) { if (inner) p2_shift(tf, lx, lane, out, L2[lane]); else p2_shift(t, lx, lane, out, L2[lane]); }
                if (pass == 2 && ph == 1) { if (inner) p2_current(tf, lx, lane, out, L2.data()); else p2_current(t, lx, lane, out, L2.data()); }
              }
          }
        }
    }
    for (int st : {(int)ST_SHIFT1, (int)ST_ZERO}) {
      if (st == ST_SHIFT1 && !ar) continue;
      if (st == ST_ZERO && !mw) continue;
      for (int x0 = 0; x0 < nx; x0 += TX)
        for (int r0 = 0; r0 < nr; r0 += TR) {
          Tile<R, M, false, false> t = pass_tile_at(n, x0, r0);
          t.g.TX = TX; t.g.TR = TR;
          for (int tid = 0; tid < nthreads; tid++) run_stage<R, M, false, false>(t, st, tid, nthreads);
        }
    }
  }
  // flat stage passes (fused == 3): blocks of 256 consecutive points in
  // (x, r) order, each point a 1 x 1 tile
  // (fused == 4: the same, one (point, mode) per thread in the
  // mode-independent passes)
  for (int n = 0; n < nsteps && (fused == 3 || fused == 4); n++) {
    const bool ax = (flags & (F_AXION | F_AREM)) != 0, ar = (flags & F_AREM) != 0, mw = (flags & F_MOVING_WINDOW) != 0;
    const bool per_ = (flags & F_X_PERIODIC) != 0;
    const int order[] = {ST_LEAP0, ST_SOURCE, ST_SHIFT0, ST_CURRENT, ST_SHIFT1, ST_ZERO};
    for (int st : order) {
      if (st == ST_SOURCE && !ax) continue;
      if ((st == ST_CURRENT || st == ST_SHIFT1) && !ar) continue;
      if (st == ST_ZERO && !mw) continue;
      const bool per_mode = fused == 4 && st != ST_SOURCE && st != ST_CURRENT;
      for (int kk = 0; kk < (per_mode ? M : 1); kk++)
      for (int q0 = 0; q0 < nx * nr; q0 += 256) {
        const int cnt = std::min(256, nx * nr - q0);
        const int w0 = q0 / nr, w1 = (q0 + cnt - 1) / nr;
        const bool inner = per_ ? (nx >= (w1 - w0 + 1) + 4) : (w0 >= 2 && w1 + 3 <= nx - 1);
        for (int q = q0; q < q0 + cnt; q++) {
          Tile<R, M, false, false> t = pass_tile_at(n, q / nr, q % nr);
          t.g.TX = 1; t.g.TR = 1;
          if (per_mode) { t.k_lo = kk; t.k_hi = kk + 1; }
          if (inner) {
            Tile<R, M, false, true> tf;
            std::memcpy((void *)&tf, (const void *)&t, sizeof t);
            run_stage<R, M, false, true>(tf, st, 0, 1);
          } else {
            run_stage<R, M, false, false>(t, st, 0, 1);
          }
        }
      }
    }
  }
  for (int n = 0; n < nsteps && fused == 2; n++) {
    // stage passes: every stage over every tile before the next stage
    const int par = n & 1;
    const bool ax = (flags & (F_AXION | F_AREM)) != 0, ar = (flags & F_AREM) != 0, mw = (flags & F_MOVING_WINDOW) != 0;
    const int order[] = {ST_LEAP0, ST_SOURCE, ST_SHIFT0, ST_PHI, ST_CURRENT, ST_LEAP1, ST_SHIFT1, ST_ZERO};
    for (int st : order) {
      if ((st == ST_SOURCE || st == ST_PHI) && !ax) continue;
      if ((st == ST_CURRENT || st == ST_LEAP1 || st == ST_SHIFT1) && !ar) continue;
      if (st == ST_ZERO && !mw) continue;
      for (int x0 = 0; x0 < nx; x0 += TX)
        for (int r0 = 0; r0 < nr; r0 += TR) {
          const bool per_ = (flags & F_X_PERIODIC) != 0;
          const bool inner = per_ ? (nx >= TX + 4) : (x0 >= 2 && x0 + TX + 2 <= nx - 1);
          Tile<R, M, false, false> t;
          t.bind(I, &I);
          t.nx = nx; t.nr = nr; t.J = nr - 1;
          t.x0 = x0; t.r0 = r0;
          t.per = (flags & F_X_PERIODIC) != 0;
          t.closed = (flags & F_R_CLOSED) != 0;
          t.mw = mw;
          t.s = t.mw ? n % nx : 0;
          t.P = P;
          t.o = buf[par].data();
          t.n = buf[par ^ 1].data();
          t.h = I.h; t.dr = I.dr; t.ih = I.inv_h; t.idr = I.inv_dr;
          t.g = geo;
          t.L = L;
          t.sm = nullptr;
          t.scr = scratch.data();
          t.state_len = E;
          t.sm_len = 0;
          if (inner) {
            Tile<R, M, false, true> tf;
            std::memcpy((void *)&tf, (const void *)&t, sizeof t);
            for (int tid = 0; tid < nthreads; tid++) run_stage<R, M, false, true>(tf, st, tid, nthreads);
          } else {
            for (int tid = 0; tid < nthreads; tid++) run_stage<R, M, false, false>(t, st, tid, nthreads);
          }
        }
    }
  }
  for (int n = 0; n < nsteps && fused == 1; n++) {
    const int par = n & 1;
    for (int x0 = 0; x0 < nx; x0 += TX)
      for (int r0 = 0; r0 < nr; r0 += TR) {
        Tile<R, M, true> t;
        t.bind(I, &I);
        t.nx = nx; t.nr = nr; t.J = nr - 1;
        t.x0 = x0; t.r0 = r0;
        t.per = (flags & F_X_PERIODIC) != 0;
        t.closed = (flags & F_R_CLOSED) != 0;
        t.mw = (flags & F_MOVING_WINDOW) != 0;
        t.s = t.mw ? n % nx : 0;
        t.P = P;
        t.o = buf[par].data();
        t.n = buf[par ^ 1].data();
        t.h = I.h; t.dr = I.dr; t.ih = I.inv_h; t.idr = I.inv_dr;
        t.g = geo;
        t.L = L;
        // poison shared memory so that a read of a slot no stage wrote shows up
        for (auto &z : sm) z = mk<R>((R)1e30, (R)1e30);
        t.sm = sm.data();
        t.scr = nullptr;
        t.state_len = E;
        t.sm_len = L.total;
        for (int st = 0; st < N_STAGE; st++)
          for (int tid = 0; tid < nthreads; tid++) run_stage<R, M, true>(t, st, tid, nthreads);
      }
  }
  // export in window order
  const auto &b = buf[nsteps & 1];
  const int s = (flags & F_MOVING_WINDOW) ? nsteps % nx : 0;
  for (size_t q = 0; q < E; q++) {
    double sc_ = 1.0;
    size_t from;
    if (q < (size_t)NFIELD * P) {
      int f = (int)(q / P);
      if (f == PHI || f == TAP || f == TAM) sc_ = 1.0 / s_ax;
      else if (f >= TRP1) sc_ = 1.0 / s_ar;
      size_t rem = q % P;
      int j = (int)(rem % nr);
      size_t kw = rem / nr;
      int w = (int)(kw % nx), k = (int)(kw / nx);
      int sl = (w + s) % nx;
      from = (size_t)f * P + ((size_t)k * nx + sl) * nr + j;
    } else {
      sc_ = 1.0 / s_ax;
      size_t rem = q - (size_t)NFIELD * P;
      int w = (int)(rem % nx), k = (int)(rem / nx);
      from = (size_t)NFIELD * P + (size_t)k * nx + (w + s) % nx;
    }
    out[2 * q] = (double)b[from].re * sc_;
    out[2 * q + 1] = (double)b[from].im * sc_;
  }
}

template <class R>
int dispatch(int M, const double *canon, double *out, int nx, int nr, double h, double dr, double m_a, double g,
             uint32_t flags, const double *jx, const double *jr, const double *jt, const double *sext, int nsteps,
             int TX, int TR, int nth, int fused) {
  switch (M) {
    case 1: emu_steps<R, 1>(canon, out, nx, nr, h, dr, m_a, g, flags, jx, jr, jt, sext, nsteps, TX, TR, nth, fused); return 0;
    case 2: emu_steps<R, 2>(canon, out, nx, nr, h, dr, m_a, g, flags, jx, jr, jt, sext, nsteps, TX, TR, nth, fused); return 0;
    case 3: emu_steps<R, 3>(canon, out, nx, nr, h, dr, m_a, g, flags, jx, jr, jt, sext, nsteps, TX, TR, nth, fused); return 0;
    case 4: emu_steps<R, 4>(canon, out, nx, nr, h, dr, m_a, g, flags, jx, jr, jt, sext, nsteps, TX, TR, nth, fused); return 0;
  }
  return 1;
}

}  // namespace

extern "C" int qds_emu_steps(int M, const double *canon, double *out, int nx, int nr, double h, double dr,
                             double m_a, double g, uint32_t flags, const double *jx, const double *jr,
                             const double *jt, const double *sext, int nsteps, int TX, int TR, int nthreads,
                             int fused) {
  if (flags & F_FP32)
    return dispatch<float>(M, canon, out, nx, nr, h, dr, m_a, g, flags, jx, jr, jt, sext, nsteps, TX, TR, nthreads, fused);
  return dispatch<double>(M, canon, out, nx, nr, h, dr, m_a, g, flags, jx, jr, jt, sext, nsteps, TX, TR, nthreads, fused);
}

// ---------------------------------------------------------------------------
// Host emulation of the adjoint step (qds_adjoint.cuh), for CPU tests only.
#include "qds_adjoint.cuh"

namespace {

template <class R, int M>
void emu_adjoint(const double *fwd, const double *lam_new, double *lam_old, int nx, int nr, double h, double dr,
                 double m_a, double g, uint32_t flags, const double *jx, const double *jt, double *dg) {
  const size_t P = plane_elems(M, nx, nr), E = state_elems(M, nx, nr);
  std::vector<C<R>> F(E), LN(E), LO(E), SB((size_t)N_SB * P);
  for (size_t q = 0; q < E; q++) {
    F[q] = mk<R>((R)fwd[2 * q], (R)fwd[2 * q + 1]);
    LN[q] = mk<R>((R)lam_new[2 * q], (R)lam_new[2 * q + 1]);
    LO[q] = mk<R>((R)1e30, (R)1e30);  // every entry must be written
  }
  std::vector<C<R>> sjx, sjt;
  if (jx) { sjx.resize(P); for (size_t q = 0; q < P; q++) sjx[q] = mk<R>((R)jx[2 * q], (R)jx[2 * q + 1]); }
  if (jt) { sjt.resize(P); for (size_t q = 0; q < P; q++) sjt[q] = mk<R>((R)jt[2 * q], (R)jt[2 * q + 1]); }
  Inst<R> I;
  std::memset(&I, 0, sizeof I);
  I.nx = nx; I.nr = nr; I.M = M; I.flags = flags;
  I.h = (R)h; I.dr = (R)dr; I.inv_h = (R)(1.0 / h); I.inv_dr = (R)(1.0 / dr);
  I.ma2 = (R)(m_a * m_a);
  I.gs = (R)g; I.gj = (R)g;
  I.jx = jx ? sjx.data() : nullptr;
  I.jt = jt ? sjt.data() : nullptr;
  Adj<R, M> a;
  Tile<R, M, false, false> &t = a.f;
  t.bind(I, &I);
  t.nx = nx; t.nr = nr; t.J = nr - 1; t.x0 = 0; t.r0 = 0; t.s = 0;
  t.per = false; t.closed = false; t.mw = false;
  t.P = P; t.o = F.data(); t.n = nullptr;
  t.h = I.h; t.dr = I.dr; t.ih = I.inv_h; t.idr = I.inv_dr;
  t.sm = nullptr; t.scr = nullptr;
  t.cw = -(1 << 28);  // set per column below
  t.state_len = E; t.sm_len = 0;
  a.ln = LN.data(); a.lo = LO.data(); a.sb = SB.data(); a.dg = dg;
  a.nx = nx; a.nr = nr; a.J = nr - 1; a.P = P;
  a.mw = (flags & F_MOVING_WINDOW) != 0;
  a.h = I.h; a.dr = I.dr; a.ih = I.inv_h; a.idr = I.inv_dr;
  a.gs = I.gs; a.ma2 = I.ma2;
  double acc = 0;
  for (int st = 0; st < N_ADSTAGE; st++)
    for (int w = 0; w < nx; w++) {
      a.f.set_point(w);
      for (int j = 0; j < nr; j++) adj_point<R, M>(a, st, w, j, acc);
    }
  if (dg) *dg += acc;
  for (size_t q = 0; q < E; q++) {
    lam_old[2 * q] = (double)LO[q].re;
    lam_old[2 * q + 1] = (double)LO[q].im;
  }
}

}  // namespace

extern "C" int qds_emu_adjoint(int M, const double *fwd, const double *lam_new, double *lam_old, int nx, int nr,
                               double h, double dr, double m_a, double g, uint32_t flags, const double *jx,
                               const double *jt, double *dg) {
  const bool f32 = (flags & F_FP32) != 0;
  switch (M) {
#define QDS_EMU_ADJ(MM)                                                                              \
  case MM:                                                                                           \
    if (f32) emu_adjoint<float, MM>(fwd, lam_new, lam_old, nx, nr, h, dr, m_a, g, flags, jx, jt, dg); \
    else emu_adjoint<double, MM>(fwd, lam_new, lam_old, nx, nr, h, dr, m_a, g, flags, jx, jt, dg);    \
    return 0;
    QDS_EMU_ADJ(1) QDS_EMU_ADJ(2) QDS_EMU_ADJ(3) QDS_EMU_ADJ(4)
#undef QDS_EMU_ADJ
  }
  return 1;
}
