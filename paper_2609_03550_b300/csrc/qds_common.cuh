// qds_common.cuh -- types shared by the QDS field-step kernels.
//
// Complex azimuthal-mode planes (Sec. 2, Eq. fourier_decomp), stored
// interleaved (re, im) with the radial index fastest: plane[m][x][r].  One
// instance's state is two ping-pong copies of
//   15 planes  Trp Trm Ttp Ttm Ex Bx phi Tap Tam Trp1 Trm1 Ttp1 Ttm1 Ex1 Bx1
//   + phi_prev[m][x]  (phi on the outermost half row one step back)
// in the working precision R (float or double).
#pragma once

#include <cmath>
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

template <class R>
QDS_HD bool finite_c(C<R> a) {
#if defined(__CUDA_ARCH__)
  return isfinite(a.re) && isfinite(a.im);
#else
  return std::isfinite(a.re) && std::isfinite(a.im);
#endif
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

// Per-instance descriptor (device resident).  ld is the row stride of a
// plane (nr, rounded up to even in FP32 so that every column starts on a
// 16-byte boundary for the bulk tensor copies); rows nr..ld-1 are padding.
template <class R>
struct Inst {
  int nx, nr, ld, M;
  uint32_t flags;
  R h, dr, inv_h, inv_dr;
  R ma2;        // m_a^2
  R gs;         // coupling in the axion source term of Gamma_a
  R gj;         // coupling in the axion current j_a
  C<R> *state[2];        // ping-pong bases: 15 planes, then phi_prev
  C<R> *scratch;         // pass mode: Gamma_a, j_a,x, j_a,r, j_a,th planes
  const C<R> *jx, *jr, *jt, *sext;  // optional sources [M][nx][nr]
  long long sstride;                // elements between the sources of consecutive steps (0: the same every step)
  // optional laser injection at x_min: the inflow T_r^+, T_th^- of the
  // exterior cell behind x_min, [M][nr] each, istride elements apart from
  // step to step (0: the same every step)
  const C<R> *in_rp, *in_tm;
  long long istride;
};

// Row stride of the working layout for precision R.
template <class R>
QDS_HD int row_stride(int nr) { return sizeof(R) == 4 ? nr + (nr & 1) : nr; }
// Elements of one field plane set [M][nx][ld] and of one copy of the state
// (15 plane sets, then phi_prev[M][nx]).
QDS_HD size_t plane_elems(int M, int nx, int ld) { return (size_t)M * nx * ld; }
QDS_HD size_t state_elems(int M, int nx, int ld) {
  return (size_t)NFIELD * plane_elems(M, nx, ld) + (size_t)M * nx;
}

}  // namespace qds
