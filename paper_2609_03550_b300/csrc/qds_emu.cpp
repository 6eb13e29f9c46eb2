#include <algorithm>
// qds_emu.cpp -- host emulation of the step kernels, for CPU tests only.
//
// Compiles the same stage code as the CUDA kernels (qds_stages.cuh,
// qds_march.cuh) for the host with bounds checks on the shared-memory and
// global accesses, and runs each CTA's stages in kernel order (all threads
// of a stage before the next stage), the bulk tensor copies replaced by
// copies with the same zero fill.  It exists so that the indexing can be
// checked on the CPU before the kernels run on a GPU; it is a separate
// library (libqds_emu.so) that the product path never loads.
#define QDS_EMU 1
#include <array>
#include <cstring>
#include <vector>

#include "qds_march.cuh"

using namespace qds;

namespace {

template <class R, int M>
struct EmuState {
  int nx, nr, ld;
  size_t P, E;
  std::vector<C<R>> buf[2], scratch;
};

// Flat stage passes: blocks of 256 consecutive points in (x, r) order, each
// point a 1 x 1 tile, unchecked where the block's x-halo is inside the window.
template <class R, int M>
void emu_flat_step(EmuState<R, M> &S, const Inst<R> &I, int n, uint32_t flags) {
  const int nx = S.nx, nr = S.nr;
  const bool ax = (flags & (F_AXION | F_AREM)) != 0, ar = (flags & F_AREM) != 0, mw = (flags & F_MOVING_WINDOW) != 0;
  const bool per_ = (flags & F_X_PERIODIC) != 0;
  for (int st = 0; st < N_STAGE; st++) {
    if (st == ST_SOURCE && !ax) continue;
    if ((st == ST_CURRENT || st == ST_SHIFT1) && !ar) continue;
    if (st == ST_ZERO && !mw) continue;
    for (int q0 = 0; q0 < nx * nr; q0 += 256) {
      const int cnt = std::min(256, nx * nr - q0);
      const int w0 = q0 / nr, w1 = (q0 + cnt - 1) / nr;
      const bool inner = per_ ? (nx >= (w1 - w0 + 1) + 4) : (w0 >= 2 && w1 + 3 <= nx - 1);
      for (int q = q0; q < q0 + cnt; q++) {
        Tile<R, M, false> t;
        t.bind(I, &I);
        t.nx = nx; t.nr = nr; t.ld = S.ld; t.J = nr - 1;
        t.x0 = q / nr; t.r0 = q % nr;
        t.per = per_;
        t.closed = (flags & F_R_CLOSED) != 0;
        t.mw = mw;
        t.s = t.mw ? n % nx : 0;
        t.P = S.P;
        t.o = S.buf[n & 1].data();
        t.n = S.buf[(n & 1) ^ 1].data();
        t.h = I.h; t.dr = I.dr; t.ih = I.inv_h; t.idr = I.inv_dr;
        t.scr = S.scratch.data();
        t.state_len = S.E;
        if (inner) {
          Tile<R, M, true> tf;
          std::memcpy((void *)&tf, (const void *)&t, sizeof t);
          run_stage<R, M, true>(tf, st);
        } else {
          run_stage<R, M, false>(t, st);
        }
      }
    }
  }
}

// The bulk tensor copy of one column: box [nbox planes][M][RB rows] of the
// planes f0.. of base (stride P), rows rb0.., column coordinate coord;
// coordinates outside (rows < 0 or >= nr, coord >= nx) read as zero.
template <class R, int M>
void emu_copy_box(const EmuState<R, M> &S, const C<R> *base, int f0, int nbox, int coord, int rb0, int RB,
                  C<R> *dst) {
  for (int f = 0; f < nbox; f++)
    for (int k = 0; k < M; k++)
      for (int r = 0; r < RB; r++) {
        const int row = rb0 + r;
        C<R> v = zero<R>();
        if (coord >= 0 && coord < S.nx && row >= 0 && row < S.nr)
          v = base[(size_t)(f0 + f) * S.P + ((size_t)k * S.nx + coord) * S.ld + row];
        dst[(f * M + k) * RB + r] = v;
      }
}

// One x-marching kernel (KIND 0: EM + axion + j_a, 1: regenerated EM) over
// all its work items, CTA by CTA, every phase over all threads of the CTA
// before the next (the kernel's barriers), the ring filled as the bulk
// copies would fill it.  The shared memory is poisoned with NaN (with NaN
// guard regions on both sides), so that a read of anything no copy or phase
// wrote shows up in the result.
template <class R, int M, int RB, int KIND>
void emu_march_kernel(EmuState<R, M> &S, const Inst<R> &I0, int n, uint32_t flags, int seg) {
  using Sh = MarchShape<R, M, RB, KIND>;
  const int nx = S.nx, nr = S.nr;
  const MarchGeo geo = march_geo<R>(KIND, M, RB);
  const int halo = KIND == 0 ? kHalo1 : kHalo2;
  const size_t guard = 8192;
  std::vector<C<R>> smv(geo.off_bar / sizeof(C<R>) + 1 + 2 * guard);
  C<R> *sm = smv.data() + guard;
  const bool ar = (flags & F_AREM) != 0;
  Inst<R> I = I0;
  I.state[0] = S.buf[0].data();
  I.state[1] = S.buf[1].data();
  I.scratch = S.scratch.data();
  std::vector<MarchItem> items;
  march_bands(nr, RB, halo, [&](int r0, int r1, int rb0) {
    for (int xa = 0; xa < nx; xa += seg) {
      MarchItem it{};
      it.inst = 0; it.r0 = r0; it.r1 = r1; it.rb0 = rb0; it.xa = xa; it.xb = std::min(nx, xa + seg);
      items.push_back(it);
    }
  });
  const int nth = M * RB;
  std::vector<MarchCtx<R, M, RB, KIND>> ctx(nth);
  std::vector<K1Regs<R>> regs(nth);
  std::vector<std::array<K2Hist<R>, 2>> hist(nth);
  for (const MarchItem &it : items) {
    for (auto &v : smv) v = mk<R>((R)NAN, (R)NAN);
    for (int tid = 0; tid < nth; tid++) {
      march_ctx<R, M, RB, KIND>(ctx[tid], I, it, sm, (unsigned long long)n, tid);
      ctx[tid].jx = I.jx; ctx[tid].jr = I.jr; ctx[tid].jt = I.jt; ctx[tid].sext = I.sext;
      ctx[tid].in_rp = I.in_rp; ctx[tid].in_tm = I.in_tm;
      ctx[tid].state_len = S.E;
      regs[tid].gam_prev = regs[tid].gam = regs[tid].tap_prev = regs[tid].tam_prev = zero<R>();
      regs[tid].bad = false;
      const C<R> nan = mk<R>((R)NAN, (R)NAN);
      for (int q = 0; q < 2; q++) hist[tid][q] = K2Hist<R>{nan, nan, nan, nan, nan, nan, nan, nan, nan, nan};
    }
    const MarchCtx<R, M, RB, KIND> &c0 = ctx[0];
    const int L0 = c0.L0, L1 = march_last(KIND, it.xb), C1 = march_last_col(KIND, it.xb);
    auto load = [&](int col) {
      C<R> *slot = sm + ((col - L0) % Sh::NS) * Sh::SS;
      const int coord = march_coord(col, nx, c0.s, c0.per);
      if (KIND == 0) {
        emu_copy_box<R, M>(S, c0.o, 0, 9, coord, it.rb0, RB, slot);
      } else {
        emu_copy_box<R, M>(S, c0.o, TRP1, 6, coord, it.rb0, RB, slot);
        emu_copy_box<R, M>(S, S.scratch.data(), 1, 3, coord, it.rb0, RB, slot + 6 * M * RB);
      }
    };
    // the copies land when the kernel issues them (three ahead, then one
    // per iteration after its last phase), no later than they are read
    for (int col = L0; col <= C1 && col < L0 + 3; col++) load(col);
    bool bad = false;
    for (int L = L0; L <= L1; L++) {
      for (int tid = 0; tid < nth; tid++) ctx[tid].iter(L);
      if constexpr (KIND == 0) {
        // the boundary warp (lane k: the outer half row of mode k) works in
        // the same phases as the main threads; its writes do not overlap theirs
        for (int tid = 0; tid < nth; tid++) k1_inflow<R, M, RB>(ctx[tid], L);
        for (int tid = 0; tid < nth; tid++) k1_p1<R, M, RB>(ctx[tid], L);
        for (int k = 0; k < M; k++) {
          const int t = k * RB + (nr - 1 - it.rb0);
          if (nr - 1 - it.rb0 < RB && outer_active<R, M, RB>(ctx[t])) outer_p1<R, M, RB>(ctx[t], L);
        }
        for (int tid = 0; tid < nth; tid++) k1_p2<R, M, RB>(ctx[tid], L, ar);
        for (int tid = 0; tid < nth; tid++) k1_p3<R, M, RB>(ctx[tid], L, regs[tid]);
        for (int k = 0; k < M; k++) {
          const int t = k * RB + (nr - 1 - it.rb0);
          if (nr - 1 - it.rb0 < RB && outer_active<R, M, RB>(ctx[t])) (void)outer_p3<R, M, RB>(ctx[t], L);
        }
      } else {
        for (int tid = 0; tid < nth; tid++) k2_p1<R, M, RB>(ctx[tid], L);
        for (int tid = 0; tid < nth; tid++) {
          K2Hist<R>(&h)[2] = *reinterpret_cast<K2Hist<R>(*)[2]>(hist[tid].data());
          k2_p2<R, M, RB>(ctx[tid], L, h, bad);
        }
      }
      if (L + 3 <= C1) load(L + 3);
    }
  }
}

// The ring heights the kernels are compiled for.
template <class R, int M, int KIND>
bool emu_march_rb(EmuState<R, M> &S, const Inst<R> &I, int n, uint32_t flags, int RB, int seg) {
  switch (RB) {
    case 8: emu_march_kernel<R, M, 8, KIND>(S, I, n, flags, seg); return true;
    case 16: emu_march_kernel<R, M, 16, KIND>(S, I, n, flags, seg); return true;
    case 24: emu_march_kernel<R, M, 24, KIND>(S, I, n, flags, seg); return true;
    case 32: emu_march_kernel<R, M, 32, KIND>(S, I, n, flags, seg); return true;
    case 64: emu_march_kernel<R, M, 64, KIND>(S, I, n, flags, seg); return true;
  }
  return false;
}

// mode 0: flat stage passes; mode 1: the x-marching kernels with rows per
// CTA RB1 (first kernel), RB2 (second) and seg columns per CTA.
template <class R, int M>
void emu_steps(const double *canon, double *out, int nx, int nr, double h, double dr, double m_a, double g,
               uint32_t flags, const double *jx, const double *jr, const double *jt, const double *sext,
               const double *in_rp, const double *in_tm, long long istride, int nsteps, int RB1, int RB2, int seg,
               int mode) {
  EmuState<R, M> S;
  S.nx = nx; S.nr = nr; S.ld = row_stride<R>(nr);
  const int ld = S.ld;
  S.P = plane_elems(M, nx, ld);
  S.E = state_elems(M, nx, ld);
  const size_t P = S.P, Pc = plane_elems(M, nx, nr), Ec = state_elems(M, nx, nr);
  const bool sc = (flags & (F_FP32 | F_SCALE_G)) && g != 0.0;
  const double s_ax = sc ? 1.0 / g : 1.0, s_ar = sc ? 1.0 / (g * g) : 1.0;
  S.buf[0].assign(S.E, zero<R>());
  S.buf[1].assign(S.E, zero<R>());
  for (size_t q = 0; q < Ec; q++) {
    double sc_ = 1.0;
    size_t to;
    if (q < (size_t)NFIELD * Pc) {
      const int f = (int)(q / Pc);
      if (f == PHI || f == TAP || f == TAM) sc_ = s_ax;
      else if (f >= TRP1) sc_ = s_ar;
      const size_t rem = q % Pc;
      to = (size_t)f * P + (rem / nr) * ld + rem % nr;
    } else {
      sc_ = s_ax;
      to = (size_t)NFIELD * P + (q - (size_t)NFIELD * Pc);
    }
    S.buf[0][to] = S.buf[1][to] = mk<R>((R)(canon[2 * q] * sc_), (R)(canon[2 * q + 1] * sc_));
  }
  std::vector<C<R>> sj[4];
  const double *srcs[4] = {jx, jr, jt, sext};
  for (int a = 0; a < 4; a++)
    if (srcs[a]) {
      sj[a].resize(Pc);
      for (size_t q = 0; q < Pc; q++) sj[a][q] = mk<R>((R)srcs[a][2 * q], (R)srcs[a][2 * q + 1]);
    }
  Inst<R> I;
  std::memset(&I, 0, sizeof I);
  I.nx = nx; I.nr = nr; I.ld = ld; I.M = M; I.flags = flags;
  I.h = (R)h; I.dr = (R)dr; I.inv_h = (R)(1.0 / h); I.inv_dr = (R)(1.0 / dr);
  I.ma2 = (R)(m_a * m_a);
  I.gs = sc ? (R)1 : (R)g;
  I.gj = sc ? (R)1 : (R)g;
  I.jx = jx ? sj[0].data() : nullptr;
  I.jr = jr ? sj[1].data() : nullptr;
  I.jt = jt ? sj[2].data() : nullptr;
  I.sext = sext ? sj[3].data() : nullptr;
  S.scratch.assign(4 * P, mk<R>((R)1e30, (R)1e30));
  const bool ar = (flags & F_AREM) != 0;
  const size_t nin = (size_t)M * nr;
  std::vector<C<R>> irp(nin), itm(nin);
  for (int n = 0; n < nsteps; n++) {
    // injection at x_min of step n (istride complex elements per step)
    I.in_rp = I.in_tm = nullptr;
    for (size_t q = 0; q < nin; q++) {
      if (in_rp) irp[q] = mk<R>((R)in_rp[2 * (n * istride + q)], (R)in_rp[2 * (n * istride + q) + 1]);
      if (in_tm) itm[q] = mk<R>((R)in_tm[2 * (n * istride + q)], (R)in_tm[2 * (n * istride + q) + 1]);
    }
    if (in_rp) I.in_rp = irp.data();
    if (in_tm) I.in_tm = itm.data();
    if (mode == 0) {
      emu_flat_step<R, M>(S, I, n, flags);
    } else {
      if (!emu_march_rb<R, M, 0>(S, I, n, flags, RB1, seg)) std::abort();
      if (ar && !emu_march_rb<R, M, 1>(S, I, n, flags, RB2, seg)) std::abort();
    }
  }
  // export in window order
  const auto &b = S.buf[nsteps & 1];
  const int s = (flags & F_MOVING_WINDOW) ? nsteps % nx : 0;
  for (size_t q = 0; q < Ec; q++) {
    double sc_ = 1.0;
    size_t from;
    if (q < (size_t)NFIELD * Pc) {
      int f = (int)(q / Pc);
      if (f == PHI || f == TAP || f == TAM) sc_ = 1.0 / s_ax;
      else if (f >= TRP1) sc_ = 1.0 / s_ar;
      size_t rem = q % Pc;
      int j = (int)(rem % nr);
      size_t kw = rem / nr;
      int w = (int)(kw % nx), k = (int)(kw / nx);
      int sl = (w + s) % nx;
      from = (size_t)f * P + ((size_t)k * nx + sl) * ld + j;
    } else {
      sc_ = 1.0 / s_ax;
      size_t rem = q - (size_t)NFIELD * Pc;
      int w = (int)(rem % nx), k = (int)(rem / nx);
      from = (size_t)NFIELD * P + (size_t)k * nx + (w + s) % nx;
    }
    out[2 * q] = (double)b[from].re * sc_;
    out[2 * q + 1] = (double)b[from].im * sc_;
  }
}

template <class R>
int dispatch(int M, const double *canon, double *out, int nx, int nr, double h, double dr, double m_a, double g,
             uint32_t flags, const double *jx, const double *jr, const double *jt, const double *sext,
             const double *in_rp, const double *in_tm, long long istride, int nsteps, int RB1, int RB2, int seg,
             int mode) {
#define QDS_EMU_CASE(MM)                                                                                 \
  case MM:                                                                                               \
    emu_steps<R, MM>(canon, out, nx, nr, h, dr, m_a, g, flags, jx, jr, jt, sext, in_rp, in_tm, istride, \
                     nsteps, RB1, RB2, seg, mode);                                                       \
    return 0;
  switch (M) { QDS_EMU_CASE(1) QDS_EMU_CASE(2) QDS_EMU_CASE(3) QDS_EMU_CASE(4) }
#undef QDS_EMU_CASE
  return 1;
}

}  // namespace

// mode 0: flat stage passes; 1: x-marching kernels (rows RB1, RB2 per CTA,
// seg columns per CTA).  in_rp / in_tm: laser injection at x_min ([M][nr]
// complex per step, istride complex elements apart; may be NULL).
extern "C" int qds_emu_steps_inflow(int M, const double *canon, double *out, int nx, int nr, double h, double dr,
                                    double m_a, double g, uint32_t flags, const double *jx, const double *jr,
                                    const double *jt, const double *sext, const double *in_rp,
                                    const double *in_tm, long long istride, int nsteps, int RB1, int RB2, int seg,
                                    int mode) {
  auto ok_rb = [](int rb) { return rb == 8 || rb == 16 || rb == 24 || rb == 32 || rb == 64; };
  if (!ok_rb(RB1) || !ok_rb(RB2) || seg < 1 || istride < 0) return 2;
  if (flags & F_FP32)
    return dispatch<float>(M, canon, out, nx, nr, h, dr, m_a, g, flags, jx, jr, jt, sext, in_rp, in_tm, istride,
                           nsteps, RB1, RB2, seg, mode);
  return dispatch<double>(M, canon, out, nx, nr, h, dr, m_a, g, flags, jx, jr, jt, sext, in_rp, in_tm, istride,
                          nsteps, RB1, RB2, seg, mode);
}

extern "C" int qds_emu_steps(int M, const double *canon, double *out, int nx, int nr, double h, double dr,
                             double m_a, double g, uint32_t flags, const double *jx, const double *jr,
                             const double *jt, const double *sext, int nsteps, int RB1, int RB2, int seg,
                             int mode) {
  return qds_emu_steps_inflow(M, canon, out, nx, nr, h, dr, m_a, g, flags, jx, jr, jt, sext, nullptr, nullptr, 0,
                              nsteps, RB1, RB2, seg, mode);
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
  I.nx = nx; I.nr = nr; I.ld = nr; I.M = M; I.flags = flags;
  I.h = (R)h; I.dr = (R)dr; I.inv_h = (R)(1.0 / h); I.inv_dr = (R)(1.0 / dr);
  I.ma2 = (R)(m_a * m_a);
  I.gs = (R)g; I.gj = (R)g;
  I.jx = jx ? sjx.data() : nullptr;
  I.jt = jt ? sjt.data() : nullptr;
  Adj<R, M> a;
  Tile<R, M, false> &t = a.f;
  t.bind(I, &I);
  t.nx = nx; t.nr = nr; t.ld = nr; t.J = nr - 1; t.x0 = 0; t.r0 = 0; t.s = 0;
  t.per = false; t.closed = false; t.mw = false;
  t.P = P; t.o = F.data(); t.n = nullptr;
  t.h = I.h; t.dr = I.dr; t.ih = I.inv_h; t.idr = I.inv_dr;
  t.scr = nullptr;
  t.cw = -(1 << 28);  // set per column below
  t.state_len = E;
  a.fnext = nullptr;  // E_x, B_x^(n+1/2) recomputed
  a.ln = LN.data(); a.lo = LO.data(); a.sb = SB.data(); a.dg = dg;
  a.nx = nx; a.nr = nr; a.J = nr - 1; a.P = (unsigned)P;
  a.mw = (flags & F_MOVING_WINDOW) != 0;
  a.zero_regen = true;
  a.h = I.h; a.dr = I.dr; a.ih = I.inv_h; a.idr = I.inv_dr;
  a.gs = I.gs; a.ma2 = I.ma2;
  a.set_consts();
  double acc = 0;
  for (int st = 0; st < N_ADSTAGE; st++)
    for (int k = 0; k < (st == AD_SRC ? 1 : M); k++)
      for (int w = 0; w < nx; w++) {
        a.f.set_point(w);
        for (int j = 0; j < nr; j++) adj_point<R, M>(a, st, k, w, j, acc);
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
