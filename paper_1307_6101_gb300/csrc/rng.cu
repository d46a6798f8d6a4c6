// Counter-based random fields for the setup: Alg. 3 starts from random test
// vectors, which the library draws on the device from a 64-bit seed.
//
// Generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC 2011) and the Box-Muller transform.  The
// logarithm is 2 atanh((m-1)/(m+1)) by its odd power series after splitting off
// the binary exponent; sine and cosine of 2 pi u are Taylor series on one
// quadrant.  Every floating-point step is an IEEE-754 double operation rounded
// to nearest (the _rn intrinsics keep the compiler from fusing a multiply and an
// add), in a fixed order, so that a host implementation of the same steps draws
// the same bits.
//
// Complex entry (field j, lexicographic site x, dof k) of level l:
//   (r0, r1, r2, r3) = Philox4x32-10(counter (x, k, j, l), key (seed lo, seed hi))
//   u1 = (((r1 r0) >> 11) + 1) 2^-53,  u2 = ((r3 r2) >> 11) 2^-53
//   entry = sqrt(-2 ln u1) (cos 2 pi u2 + i sin 2 pi u2)
#include "common.cuh"
#include "kernels.h"

namespace dd {
namespace {

constexpr double kLn2 = 0.6931471805599453;      // ln 2 rounded to double
constexpr double kHalfPi = 1.5707963267948966;   // pi / 2 rounded to double
constexpr double kSqrtHalf = 0.7071067811865476;
constexpr int kLogTerms = 13;    // s^1 .. s^25
constexpr int kTrigTerms = 13;   // theta^0 .. theta^25

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    c[1] = (uint32_t)p1;
    c[3] = (uint32_t)p0;
    c[0] = n0;
    c[2] = n2;
  }
}

// ln u for u in (0, 1]
__device__ double ln_unit(double u) {
  int e = 0;
  double m = frexp(u, &e);   // exact: m in [0.5, 1)
  if (m < kSqrtHalf) {
    m = __dmul_rn(m, 2.0);
    e -= 1;
  }
  const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double t = __dmul_rn(s, s);
  double p = __ddiv_rn(1.0, (double)(2 * kLogTerms - 1));
#pragma unroll 1
  for (int i = kLogTerms - 2; i >= 0; --i) p = __dadd_rn(__dmul_rn(p, t), __ddiv_rn(1.0, (double)(2 * i + 1)));
  return __dadd_rn(__dmul_rn(2.0, __dmul_rn(s, p)), __dmul_rn((double)e, kLn2));
}

// sin and cos of 2 pi u for u in [0, 1)
__device__ void sincos_2pi(double u, double* sn, double* cs) {
  const double v = __dmul_rn(u, 4.0);
  const double q = floor(v);
  const double th = __dmul_rn(__dsub_rn(v, q), kHalfPi);
  const double t = __dmul_rn(th, th);
  // (-1)^k / (2k+1)! and (-1)^k / (2k)!, by divisions through exact integers
  double sc[kTrigTerms], cc[kTrigTerms];
  sc[0] = 1.0;
  cc[0] = 1.0;
#pragma unroll
  for (int k = 1; k < kTrigTerms; ++k) {
    sc[k] = __ddiv_rn(-sc[k - 1], (double)((2 * k) * (2 * k + 1)));
    cc[k] = __ddiv_rn(-cc[k - 1], (double)((2 * k - 1) * (2 * k)));
  }
  double ps = sc[kTrigTerms - 1], pc = cc[kTrigTerms - 1];
#pragma unroll
  for (int k = kTrigTerms - 2; k >= 0; --k) {
    ps = __dadd_rn(__dmul_rn(ps, t), sc[k]);
    pc = __dadd_rn(__dmul_rn(pc, t), cc[k]);
  }
  const double S = __dmul_rn(th, ps), C = pc;
  switch ((int)q) {
    case 0: *sn = S; *cs = C; break;
    case 1: *sn = C; *cs = -S; break;
    case 2: *sn = -S; *cs = -C; break;
    default: *sn = -C; *cs = S; break;
  }
}

__device__ cplx<double> normal_pair(uint32_t x, uint32_t k, uint32_t j, uint32_t l, uint64_t seed) {
  uint32_t c[4] = {x, k, j, l};
  philox4x32_10(c, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
  const uint64_t a = ((((uint64_t)c[1] << 32) | c[0]) >> 11) + 1;
  const uint64_t b = (((uint64_t)c[3] << 32) | c[2]) >> 11;
  const double u1 = __dmul_rn((double)a, 0x1.0p-53);
  const double u2 = __dmul_rn((double)b, 0x1.0p-53);
  const double rho = __dsqrt_rn(__dmul_rn(-2.0, ln_unit(u1)));
  double sn, cs;
  sincos_2pi(u2, &sn, &cs);
  return cmk<double>(__dmul_rn(rho, cs), __dmul_rn(rho, sn));
}

// one thread per (site, dof) entry of field j0 + blockIdx.y, written in the level's layout
__global__ void k_draw_fields(cplx<double>* __restrict__ dst, Geom g, int n, bool fine, size_t rstride, int j0,
                              int level, uint64_t seed) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)g.V * n) return;
  int xi, k;
  if (fine) {   // [12][V], component-major
    xi = (int)(t % g.V);
    k = (int)(t / g.V);
  } else {      // [V][n]
    xi = (int)(t / n);
    k = (int)(t % n);
  }
  int c[4];
  geom_coords(g, xi, c);
  const uint32_t lex = (uint32_t)lin4(c, g.L);
  const int j = j0 + (int)blockIdx.y;
  dst[(size_t)blockIdx.y * rstride + t] = normal_pair(lex, (uint32_t)k, (uint32_t)j, (uint32_t)level, seed);
}

}  // namespace

void draw_fields(cplx<double>* dst, const Geom& g, bool fine, int n, int nfields, int j0, int level, uint64_t seed,
                 size_t rstride, cudaStream_t st) {
  if (nfields <= 0) return;
  count_launch();
  k_draw_fields<<<dim3(div_up((size_t)g.V * n, 256), nfields), 256, 0, st>>>(dst, g, n, fine, rstride, j0, level,
                                                                            seed);
}

}  // namespace dd
