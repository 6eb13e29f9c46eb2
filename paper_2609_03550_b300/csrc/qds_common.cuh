// qds_common.cuh -- types shared by the QDS field-step kernels.
//
// Complex azimuthal-mode planes (Sec. 2, Eq. fourier_decomp), stored
// interleaved (re, im) with the radial index fastest: plane[m][x][r].  One
// instance's state is two ping-pong copies of
//   15 planes  Trp Trm Ttp Ttm Ex Bx phi Tap Tam Trp1 Trm1 Ttp1 Ttm1 Ex1 Bx1
//   + phi_prev[m][x]  (phi on the outermost half row one step back)
// in the working precision R (float or double).
#pragma once

#include <cstddef>
#include <cstdint>

#if defined(__CUDACC__)
#define QDS_HD __host__ __device__ __forceinline__
#else
#define QDS_HD inline
#endif

namespace qds {

enum Field : int {
  TRP = 0, TRM, TTP, TTM, EX, BX, PHI, TAP, TAM,
  TRP1, TRM1, TTP1, TTM1, EX1, BX1, NFIELD
};

enum Flag : uint32_t {
  F_AXION = 1u, F_AREM = 2u, F_MOVING_WINDOW = 4u, F_X_PERIODIC = 8u,
  F_R_CLOSED = 16u, F_FP32 = 32u, F_SCALE_G = 64u
};

// Aligned to its size, so that one complex value moves as one 8-byte (FP32)
// or 16-byte (FP64) access.
template <class R>
struct alignas(2 * sizeof(R)) C {
  R re, im;
};

template <class R> QDS_HD C<R> mk(R a, R b) { C<R> z; z.re = a; z.im = b; return z; }
template <class R> QDS_HD C<R> zero() { return mk<R>(R(0), R(0)); }
template <class R> QDS_HD C<R> operator+(C<R> a, C<R> b) { return mk<R>(a.re + b.re, a.im + b.im); }
template <class R> QDS_HD C<R> operator-(C<R> a, C<R> b) { return mk<R>(a.re - b.re, a.im - b.im); }
template <class R> QDS_HD C<R> operator-(C<R> a) { return mk<R>(-a.re, -a.im); }
template <class R> QDS_HD C<R> operator*(C<R> a, C<R> b) {
  return mk<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class R> QDS_HD C<R> operator*(R s, C<R> a) { return mk<R>(s * a.re, s * a.im); }
template <class R> QDS_HD C<R> operator*(C<R> a, R s) { return mk<R>(s * a.re, s * a.im); }
template <class R> QDS_HD C<R> &operator+=(C<R> &a, C<R> b) { a.re += b.re; a.im += b.im; return a; }
template <class R> QDS_HD C<R> &operator-=(C<R> &a, C<R> b) { a.re -= b.re; a.im -= b.im; return a; }
template <class R> QDS_HD C<R> cj(C<R> a) { return mk<R>(a.re, -a.im); }
// i * s * a
template <class R> QDS_HD C<R> imul(R s, C<R> a) { return mk<R>(-s * a.im, s * a.re); }
// a * conj(b)
template <class R> QDS_HD C<R> mul_cj(C<R> a, C<R> b) {
  return mk<R>(a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im);
}

// FP32 on sm_100 and later: sums, differences and real scalings of complex
// values as one packed two-lane instruction (same rounding per component).
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
#define QDS_PACKED_F32 1
#endif
#if defined(QDS_PACKED_F32)
__device__ __forceinline__ float2 f2(C<float> a) { return make_float2(a.re, a.im); }
__device__ __forceinline__ C<float> cf(float2 a) { return mk<float>(a.x, a.y); }
__device__ __forceinline__ C<float> operator+(C<float> a, C<float> b) { return cf(__fadd2_rn(f2(a), f2(b))); }
__device__ __forceinline__ C<float> operator-(C<float> a, C<float> b) {
  return cf(__ffma2_rn(make_float2(-1.f, -1.f), f2(b), f2(a)));
}
__device__ __forceinline__ C<float> operator*(float s, C<float> a) { return cf(__fmul2_rn(make_float2(s, s), f2(a))); }
__device__ __forceinline__ C<float> operator*(C<float> a, float s) { return cf(__fmul2_rn(make_float2(s, s), f2(a))); }
__device__ __forceinline__ C<float> &operator+=(C<float> &a, C<float> b) { a = a + b; return a; }
__device__ __forceinline__ C<float> &operator-=(C<float> &a, C<float> b) { a = a - b; return a; }
#endif

// Per-instance descriptor (device resident).
template <class R>
struct Inst {
  int nx, nr, M;
  uint32_t flags;
  R h, dr, inv_h, inv_dr;
  R ma2;        // m_a^2
  R gs;         // coupling in the axion source term of Gamma_a
  R gj;         // coupling in the axion current j_a
  C<R> *state[2];        // ping-pong bases: 15 planes, then phi_prev
  C<R> *scratch;         // pass mode: Gamma_a, j_a,x, j_a,r, j_a,th planes
  const C<R> *jx, *jr, *jt, *sext;  // optional sources [M][nx][nr]
  int tiles_x, tiles_r;  // tile grid of this instance
  int tile_base;         // first global tile index of this instance
};

QDS_HD size_t plane_elems(int M, int nx, int nr) { return (size_t)M * nx * nr; }
QDS_HD size_t state_elems(int M, int nx, int nr) {
  return (size_t)NFIELD * plane_elems(M, nx, nr) + (size_t)M * nx;
}

// Tile geometry (cells/faces in x, rows in r) and the shared-memory regions
// of the fused step.  Region bounds are in tile-local coordinates.
struct Geo {
  int TX, TR;
  // faces [-2, TX], rows [-3, TR+2]: E_x, B_x of group 0 at n+1/2
  QDS_HD int a_x0() const { return -2; }
  QDS_HD int a_nx() const { return TX + 3; }
  QDS_HD int a_r0() const { return -3; }
  QDS_HD int a_nr() const { return TR + 6; }
  // faces [-2, TX], rows [-2, TR+1]: Gamma_a at n
  QDS_HD int g_x0() const { return -2; }
  QDS_HD int g_nx() const { return TX + 3; }
  QDS_HD int g_r0() const { return -2; }
  QDS_HD int g_nr() const { return TR + 4; }
  // cells [-1, TX], rows [-2, TR+1]: T^(n+1) of group 0 and T_a^(n+1/2)
  QDS_HD int t_x0() const { return -1; }
  QDS_HD int t_nx() const { return TX + 2; }
  QDS_HD int t_r0() const { return -2; }
  QDS_HD int t_nr() const { return TR + 4; }
  // faces [-1, TX-1], rows [-2, TR+1]: phi^(n+1)
  QDS_HD int p_x0() const { return -1; }
  QDS_HD int p_nx() const { return TX + 1; }
  QDS_HD int p_r0() const { return -2; }
  QDS_HD int p_nr() const { return TR + 4; }
  // faces [-1, TX-1], rows [-1, TR]: E_x1, B_x1 at n+1/2, j_a (x, r, theta)
  QDS_HD int j_x0() const { return -1; }
  QDS_HD int j_nx() const { return TX + 1; }
  QDS_HD int j_r0() const { return -1; }
  QDS_HD int j_nr() const { return TR + 2; }

  // complex elements per mode of each region
  QDS_HD int a_sz() const { return a_nx() * a_nr(); }
  QDS_HD int g_sz() const { return g_nx() * g_nr(); }
  QDS_HD int t_sz() const { return t_nx() * t_nr(); }
  QDS_HD int p_sz() const { return p_nx() * p_nr(); }
  QDS_HD int j_sz() const { return j_nx() * j_nr(); }
};

// Shared-memory layout (complex elements), all planes per mode contiguous.
struct Smem {
  int off_a;   // 2 planes (Ex0n, Bx0n) x M
  int off_t;   // 6 planes (Trp Trm Ttp Ttm Tap Tam at new levels) x M
  int off_p;   // 1 plane x M
  int off_j;   // 5 planes (Ex1n Bx1n jax jar jat) x M; aliases Gamma_a (1 plane x M)
  int total;
};

QDS_HD Smem smem_layout(const Geo &g, int M, uint32_t flags) {
  Smem s;
  int o = 0;
  s.off_a = o; o += 2 * M * g.a_sz();
  const bool ax = (flags & (F_AXION | F_AREM)) != 0;
  const bool ar = (flags & F_AREM) != 0;
  s.off_t = o; if (ax) o += 6 * M * g.t_sz();
  s.off_p = o; if (ax) o += M * g.p_sz();
  s.off_j = o;
  if (ax) {
    int jz = ar ? 5 * M * g.j_sz() : 0;
    int gz = M * g.g_sz();
    o += (jz > gz ? jz : gz);
  }
  s.total = o;
  return s;
}

}  // namespace qds
