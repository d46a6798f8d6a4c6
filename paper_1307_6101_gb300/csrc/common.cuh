// Shared device-side definitions for the DD-alpha-AMG CUDA library.
//
// Layouts (all device memory, owned by the library):
//   fine spinor  [rhs][12][V]         complex, component-major so that a warp's
//                                      32 consecutive sites read 32 consecutive words
//   links        [mu][9][V]           complex, U_mu(x)_{ab} at (mu*9 + a*3 + b)*V + x
//   clover       [2][36][V]           real, two packed Hermitian 6x6 blocks per site
//                                      (chirality 0 = spins 0,1; 1 = spins 2,3);
//                                      FP16 copy [2][18][V] half2, pairs of packed reals
//   coarse field [rhs][V][n]          complex, dof-contiguous per coarse site
//   coarse op    [V][9][n][n]         complex, column-major blocks: k = 0 self,
//                                      1..4 forward mu, 5..8 backward mu
// Site order on every level is hierarchical: aggregate-major, then SAP block
// within the aggregate, then site within the block, each lexicographic with
// t slowest and x fastest.  SAP blocks and aggregates are therefore
// contiguous index ranges.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <cmath>

#define DD_HD __host__ __device__ __forceinline__

template <typename T>
struct alignas(2 * sizeof(T)) cplx {
  T re, im;
};

template <typename T> DD_HD cplx<T> cmk(T a, T b) { cplx<T> c; c.re = a; c.im = b; return c; }
template <typename T> DD_HD cplx<T> czero() { return cmk<T>(T(0), T(0)); }
template <typename T> DD_HD cplx<T> operator+(cplx<T> a, cplx<T> b) { return cmk<T>(a.re + b.re, a.im + b.im); }
template <typename T> DD_HD cplx<T> operator-(cplx<T> a, cplx<T> b) { return cmk<T>(a.re - b.re, a.im - b.im); }
template <typename T> DD_HD cplx<T> operator-(cplx<T> a) { return cmk<T>(-a.re, -a.im); }
template <typename T> DD_HD cplx<T> operator*(cplx<T> a, cplx<T> b) {
  return cmk<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T> DD_HD cplx<T> operator*(T s, cplx<T> a) { return cmk<T>(s * a.re, s * a.im); }
template <typename T> DD_HD cplx<T> cconj(cplx<T> a) { return cmk<T>(a.re, -a.im); }
// conj(a) * b
template <typename T> DD_HD cplx<T> cdotc(cplx<T> a, cplx<T> b) {
  return cmk<T>(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
// acc += a * b as four fused multiply-adds (no separate product and sum: on GB300
// an FP64 multiply or add costs an FP64 pipe slot like an FMA)
template <typename T> DD_HD void cfma(cplx<T>& acc, cplx<T> a, cplx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename T> DD_HD void cfmac(cplx<T>& acc, cplx<T> a, cplx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}
// (re, im) += conj(a) * b and n2 += |a|^2, fused
template <typename T> DD_HD void cdotc_acc(T& re, T& im, cplx<T> a, cplx<T> b) {
  re = fma(a.re, b.re, re);
  re = fma(a.im, b.im, re);
  im = fma(a.re, b.im, im);
  im = fma(-a.im, b.re, im);
}
template <typename T> DD_HD void cnorm2_acc(T& n2, cplx<T> a) {
  n2 = fma(a.re, a.re, n2);
  n2 = fma(a.im, a.im, n2);
}
template <typename T> DD_HD cplx<T> times_i(cplx<T> a) { return cmk<T>(-a.im, a.re); }
template <typename T> DD_HD cplx<T> times_mi(cplx<T> a) { return cmk<T>(a.im, -a.re); }
template <typename T> DD_HD T cnorm2(cplx<T> a) { return a.re * a.re + a.im * a.im; }

template <typename To, typename From> DD_HD cplx<To> ccast(cplx<From> a) {
  return cmk<To>(static_cast<To>(a.re), static_cast<To>(a.im));
}

// Storage loads: operator data is held in the compute precision, or in FP16
// (__half = one real, __half2 = one complex or a pair of reals) and widened to
// FP32 on load.
template <typename T> DD_HD T ld_real(const T* p, size_t i) { return p[i]; }
__device__ __forceinline__ float ld_real(const __half* p, size_t i) { return __half2float(p[i]); }
template <typename T> DD_HD cplx<T> ld_cplx(const cplx<T>* p, size_t i) { return p[i]; }
__device__ __forceinline__ cplx<float> ld_cplx(const __half2* p, size_t i) {
  const float2 f = __half22float2(p[i]);
  return cmk<float>(f.x, f.y);
}

// ---------------------------------------------------------------------------
// Geometry of one level: lattice extents L, aggregate extents A and SAP block
// extents B, one of which tiles the other.  The larger is the outer tile O, the
// smaller the inner tile I; index = (lin(c/O) * nIO + lin((c%O)/I)) * vI + lin(c%I),
// so aggregates and SAP blocks are both contiguous index ranges.
struct Geom {
  int L[4];
  int A[4];
  int B[4];
  int O[4];    // outer tile
  int I[4];    // inner tile
  int nO[4];   // L / O
  int nI[4];   // O / I
  int V;       // sites
  int vA;      // sites per aggregate
  int vB;      // sites per SAP block
  int vI;      // sites per inner tile
  int nIO;     // inner tiles per outer tile
  int nAgg;    // aggregates
  int nBlk;    // SAP blocks
};

DD_HD int lin4(const int c[4], const int n[4]) { return ((c[0] * n[1] + c[1]) * n[2] + c[2]) * n[3] + c[3]; }
DD_HD void delin4(int l, const int n[4], int c[4]) {
  c[3] = l % n[3]; l /= n[3];
  c[2] = l % n[2]; l /= n[2];
  c[1] = l % n[1]; l /= n[1];
  c[0] = l;
}

DD_HD int geom_index(const Geom& g, const int c[4]) {
  int a[4], b[4], l[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    a[d] = c[d] / g.O[d];
    int r = c[d] - a[d] * g.O[d];
    b[d] = r / g.I[d];
    l[d] = r - b[d] * g.I[d];
  }
  return (lin4(a, g.nO) * g.nIO + lin4(b, g.nI)) * g.vI + lin4(l, g.I);
}

DD_HD void geom_coords(const Geom& g, int idx, int c[4]) {
  int l[4], b[4], a[4];
  int loc = idx % g.vI;
  int r = idx / g.vI;
  int blk = r % g.nIO;
  int agg = r / g.nIO;
  delin4(loc, g.I, l);
  delin4(blk, g.nI, b);
  delin4(agg, g.nO, a);
#pragma unroll
  for (int d = 0; d < 4; ++d) c[d] = (a[d] * g.nI[d] + b[d]) * g.I[d] + l[d];
}

// index of the neighbour x + dir * mu_hat (periodic wrap)
DD_HD int geom_neighbor(const Geom& g, const int c[4], int mu, int dir) {
  int n[4] = {c[0], c[1], c[2], c[3]};
  n[mu] += dir;
  if (n[mu] < 0) n[mu] += g.L[mu];
  if (n[mu] >= g.L[mu]) n[mu] -= g.L[mu];
  return geom_index(g, n);
}

// does the hop from x in direction dir*mu stay in x's tile of extent t (with wrap)?
DD_HD bool hop_internal(const Geom& g, const int c[4], int mu, int dir, const int* tile) {
  int n = c[mu] + dir;
  if (n < 0) n += g.L[mu];
  if (n >= g.L[mu]) n -= g.L[mu];
  return (n / tile[mu]) == (c[mu] / tile[mu]);
}

// SAP block colour (sum of block coordinates mod 2)
DD_HD int geom_block_colour(const Geom& g, const int c[4]) {
  return (c[0] / g.B[0] + c[1] / g.B[1] + c[2] / g.B[2] + c[3] / g.B[3]) & 1;
}

DD_HD int geom_parity(const int c[4]) { return (c[0] + c[1] + c[2] + c[3]) & 1; }

// hierarchical index of the aggregate containing coarse coordinates ca on the coarse level
DD_HD int coarse_site_of(const Geom& fine, const Geom& coarse, const int c[4]) {
  int ca[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) ca[d] = c[d] / fine.A[d];
  return geom_index(coarse, ca);
}

// ---------------------------------------------------------------------------
// Launch helpers
inline unsigned int div_up(size_t a, size_t b) { return static_cast<unsigned int>((a + b - 1) / b); }

// Term selection for operator applications used by the Galerkin construction.
enum TermSel : int {
  SEL_FULL = 0,       // the whole operator
  SEL_AGG_SELF = 1,   // site-diagonal part + hops that stay inside the aggregate
  SEL_AGG_FWD = 2,    // only the forward hop mu that leaves the aggregate
  SEL_AGG_BWD = 3,    // only the backward hop mu that leaves the aggregate
};
