// Fine-level (Wilson-clover) kernels.
//
// D psi(x) = A(x) psi(x) - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
//                                     + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu) ]
// with A(x) = (m0 + 4) + C(x), C the clover term (the operator of Sec. 1 of
// the paper, whose gamma_5-symmetry D Gamma_5 = Gamma_5 D^+ needs a chiral basis
// where Gamma_5 = diag(1, 1, -1, -1)).  In that basis
//   gamma_t = [[0, 1], [1, 0]],  gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
// so (1 -+ gamma_mu) has rank 2 in spin: each hop projects the neighbour onto a
// two-spin half spinor h, multiplies the two colour vectors of h by the link,
// and reconstructs the lower two spins from the upper two:
//   forward  (1 - gamma_t): h = up - dn,            lower = -h
//   backward (1 + gamma_t): h = up + dn,            lower = +h
//   forward  (1 - gamma_k): h = up + i sigma_k dn,  lower = -i sigma_k h
//   backward (1 + gamma_k): h = up - i sigma_k dn,  lower = +i sigma_k h
// The antiperiodic sign of the time direction multiplies the hop that wraps.
#include "common.cuh"
#include "dfloat.cuh"
#include "kernels.h"
#include "tma.cuh"

#include <cstdint>
#include <mutex>

namespace {

template <typename T>
DD_HD void isigma(int mu, const cplx<T>* v0, const cplx<T>* v1, cplx<T>* w0, cplx<T>* w1) {
  // (w0, w1) = i sigma (v0, v1), sigma = sigma_z (mu = 1), sigma_y (mu = 2), sigma_x (mu = 3)
  if (mu == 3) {
#pragma unroll
    for (int a = 0; a < 3; ++a) { w0[a] = times_i(v1[a]); w1[a] = times_i(v0[a]); }
  } else if (mu == 2) {
#pragma unroll
    for (int a = 0; a < 3; ++a) { w0[a] = v1[a]; w1[a] = -v0[a]; }
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) { w0[a] = times_i(v0[a]); w1[a] = times_mi(v1[a]); }
  }
}

template <typename T>
DD_HD void su3_mul(const cplx<T> u[9], const cplx<T> v[3], cplx<T> w[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cplx<T> s = u[a * 3 + 0] * v[0];
    cfma(s, u[a * 3 + 1], v[1]);
    cfma(s, u[a * 3 + 2], v[2]);
    w[a] = s;
  }
}

template <typename T>
DD_HD void su3_dag_mul(const cplx<T> u[9], const cplx<T> v[3], cplx<T> w[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cplx<T> s = cdotc(u[0 * 3 + a], v[0]);
    cfmac(s, u[1 * 3 + a], v[1]);
    cfmac(s, u[2 * 3 + a], v[2]);
    w[a] = s;
  }
}

// acc += (1 - gamma_mu) U psi   (forward, fwd = true)  or  (1 + gamma_mu) U^+ psi (backward)
template <typename T>
DD_HD void hop_accumulate(int mu, bool fwd, const cplx<T> u[9], const cplx<T> psi[12], cplx<T> acc[12]) {
  cplx<T> h0[3], h1[3];
  const cplx<T>* up0 = psi + 0;
  const cplx<T>* up1 = psi + 3;
  const cplx<T>* dn0 = psi + 6;
  const cplx<T>* dn1 = psi + 9;
  if (mu == 0) {
    const T s = fwd ? T(-1) : T(1);
#pragma unroll
    for (int a = 0; a < 3; ++a) { h0[a] = up0[a] + s * dn0[a]; h1[a] = up1[a] + s * dn1[a]; }
  } else {
    cplx<T> q0[3], q1[3];
    isigma(mu, dn0, dn1, q0, q1);
    if (fwd) {
#pragma unroll
      for (int a = 0; a < 3; ++a) { h0[a] = up0[a] + q0[a]; h1[a] = up1[a] + q1[a]; }
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a) { h0[a] = up0[a] - q0[a]; h1[a] = up1[a] - q1[a]; }
    }
  }
  cplx<T> g0[3], g1[3];
  if (fwd) { su3_mul(u, h0, g0); su3_mul(u, h1, g1); }
  else { su3_dag_mul(u, h0, g0); su3_dag_mul(u, h1, g1); }
#pragma unroll
  for (int a = 0; a < 3; ++a) { acc[a] = acc[a] + g0[a]; acc[3 + a] = acc[3 + a] + g1[a]; }
  if (mu == 0) {
    const T s = fwd ? T(-1) : T(1);
#pragma unroll
    for (int a = 0; a < 3; ++a) { acc[6 + a] = acc[6 + a] + s * g0[a]; acc[9 + a] = acc[9 + a] + s * g1[a]; }
  } else {
    cplx<T> q0[3], q1[3];
    isigma(mu, g0, g1, q0, q1);
    if (fwd) {
#pragma unroll
      for (int a = 0; a < 3; ++a) { acc[6 + a] = acc[6 + a] - q0[a]; acc[9 + a] = acc[9 + a] - q1[a]; }
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a) { acc[6 + a] = acc[6 + a] + q0[a]; acc[9 + a] = acc[9 + a] + q1[a]; }
    }
  }
}

// packed Hermitian 6x6: 6 real diagonals, then the 15 upper off-diagonals (row-major) as re, im
DD_HD int herm_off(int i, int j) { return i * 6 - (i * (i + 1)) / 2 + (j - i - 1); }

// Clover storage: per chirality 36 packed reals, component-major with stride V.
// FP32/FP64: one row per real ([2][36][V]); FP16: one __half2 row per pair of
// consecutive reals ([2][18][V]), so a row load brings two reals.
template <typename CS> struct ClovRows { static constexpr int per_chir = 36; };
template <> struct ClovRows<__half2> { static constexpr int per_chir = 18; };

template <typename T, typename CS>
DD_HD void load_clover36(const CS* __restrict__ a, size_t stride, T c[36]) {
#pragma unroll
  for (int i = 0; i < 36; ++i) c[i] = T(ld_real(a, (size_t)i * stride));
}
__device__ __forceinline__ void load_clover36(const __half2* __restrict__ a, size_t stride, float c[36]) {
#pragma unroll
  for (int j = 0; j < 18; ++j) {
    const float2 f = __half22float2(a[(size_t)j * stride]);
    c[2 * j] = f.x;
    c[2 * j + 1] = f.y;
  }
}

// out = (A + shift) in for the two packed Hermitian 6x6 blocks (shift on the diagonal)
template <typename T, typename CS>
DD_HD void clover_apply(const CS* __restrict__ clov, int V, int x, const cplx<T> in[12], cplx<T> out[12],
                        T shift = T(0)) {
#pragma unroll
  for (int ch = 0; ch < 2; ++ch) {
    T a[36];
    load_clover36(clov + (size_t)ch * ClovRows<CS>::per_chir * V + x, (size_t)V, a);
    const cplx<T>* v = in + 6 * ch;
    cplx<T>* w = out + 6 * ch;
#pragma unroll
    for (int i = 0; i < 6; ++i) w[i] = (a[i] + shift) * v[i];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
      for (int j = i + 1; j < 6; ++j) {
        const int p = 6 + 2 * herm_off(i, j);
        const cplx<T> e = cmk<T>(a[p], a[p + 1]);
        cfma(w[i], e, v[j]);
        cfmac(w[j], e, v[i]);
      }
    }
  }
}

template <typename T, typename LS>
DD_HD void load_link(const LS* __restrict__ U, int V, int mu, int x, cplx<T> u[9]) {
#pragma unroll
  for (int k = 0; k < 9; ++k) u[k] = ld_cplx(U, (size_t)(mu * 9 + k) * V + x);
}

// x * (+1 or -1) as a flip of the sign bit (integer operation: no FP64 pipe use; same bits as the product)
__device__ __forceinline__ double sign_flip(double x, bool neg) {
  return __longlong_as_double(__double_as_longlong(x) ^ (neg ? (long long)0x8000000000000000ULL : 0LL));
}
__device__ __forceinline__ float sign_flip(float x, bool neg) {
  return __int_as_float(__float_as_int(x) ^ (neg ? (int)0x80000000u : 0));
}

// the 12 components of a spinor at x times sign (+1 / -1); chir >= 0 keeps one chirality
template <typename T>
__device__ __forceinline__ void load_spinor(const cplx<T>* __restrict__ p, int V, int x, cplx<T> s[12], T sign,
                                            int chir) {
  const bool neg = sign < T(0);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const bool keep = chir < 0 || (k / 6) == chir;
    const cplx<T> v = p[(size_t)k * V + x];
    s[k] = keep ? cmk<T>(sign_flip(v.re, neg), sign_flip(v.im, neg)) : czero<T>();
  }
}

// ---------------------------------------------------------------------------
template <typename T, bool RESID, typename LS, typename CS>
__global__ void k_fine_dslash(cplx<T>* __restrict__ out, const cplx<T>* __restrict__ in,
                              const cplx<T>* __restrict__ bsrc, const LS* __restrict__ U,
                              const CS* __restrict__ clov, Geom g, int bc_t, size_t rstride,
                              int sel, int sel_mu, int in_chir, T shift) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.V) return;
  const size_t ro = (size_t)blockIdx.y * rstride;
  const cplx<T>* ps = in + ro;
  const int V = g.V;
  int c[4];
  geom_coords(g, x, c);
  cplx<T> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = czero<T>();
  cplx<T> nb[12], u[9];
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    const bool inf = hop_internal(g, c, mu, +1, g.A);
    const bool inb = hop_internal(g, c, mu, -1, g.A);
    bool tf = true, tb = true;
    if (sel == SEL_AGG_SELF) { tf = inf; tb = inb; }
    else if (sel == SEL_AGG_FWD) { tf = (mu == sel_mu) && !inf; tb = false; }
    else if (sel == SEL_AGG_BWD) { tf = false; tb = (mu == sel_mu) && !inb; }
    if (tf) {
      const int n = geom_neighbor(g, c, mu, +1);
      const T sgn = (mu == 0 && c[0] == g.L[0] - 1) ? T(bc_t) : T(1);
      load_spinor(ps, V, n, nb, sgn, in_chir);
      load_link(U, V, mu, x, u);
      hop_accumulate(mu, true, u, nb, acc);
    }
    if (tb) {
      const int n = geom_neighbor(g, c, mu, -1);
      const T sgn = (mu == 0 && c[0] == 0) ? T(bc_t) : T(1);
      load_spinor(ps, V, n, nb, sgn, in_chir);
      load_link(U, V, mu, n, u);
      hop_accumulate(mu, false, u, nb, acc);
    }
  }
  cplx<T> d[12];
  if (sel == SEL_FULL || sel == SEL_AGG_SELF) {
    load_spinor(ps, V, x, nb, T(1), in_chir);
    clover_apply(clov, V, x, nb, d, shift);
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) d[k] = czero<T>();
  }
  cplx<T>* po = out + ro;
  if (RESID) {
    const cplx<T>* pb = bsrc + ro;
#pragma unroll
    for (int k = 0; k < 12; ++k) po[(size_t)k * V + x] = pb[(size_t)k * V + x] - (d[k] - T(0.5) * acc[k]);
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) po[(size_t)k * V + x] = d[k] - T(0.5) * acc[k];
  }
}

// ---------------------------------------------------------------------------
// The full operator in double-FP32 arithmetic on FP64 vectors: the same hop and clover code as
// k_fine_dslash instantiated for the double-FP32 type, links and clover term (with the mass shift)
// stored as double-FP32 pairs, the FP64 input split on load and the result rounded to FP64.
__device__ __forceinline__ void load_spinor_df(const cplx<double>* __restrict__ p, int V, int x, cplx<dfl> s[12],
                                               bool neg) {
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const cplx<double> v = p[(size_t)k * V + x];
    s[k] = cmk<dfl>(df_from_double(sign_flip(v.re, neg)), df_from_double(sign_flip(v.im, neg)));
  }
}

template <bool RESID>
__global__ void __launch_bounds__(128) k_fine_dslash_df(cplx<double>* __restrict__ out,
                                                         const cplx<double>* __restrict__ in,
                                                         const cplx<double>* __restrict__ bsrc,
                                                         const cplx<dfl>* __restrict__ U,
                                                         const dfl* __restrict__ clov, Geom g, int bc_t,
                                                         size_t rstride) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.V) return;
  const size_t ro = (size_t)blockIdx.y * rstride;
  const cplx<double>* ps = in + ro;
  const int V = g.V;
  int c[4];
  geom_coords(g, x, c);
  cplx<dfl> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = czero<dfl>();
  cplx<dfl> nb[12], u[9];
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    {
      const int n = geom_neighbor(g, c, mu, +1);
      load_spinor_df(ps, V, n, nb, mu == 0 && c[0] == g.L[0] - 1 && bc_t < 0);
      load_link(U, V, mu, x, u);
      hop_accumulate(mu, true, u, nb, acc);
    }
    {
      const int n = geom_neighbor(g, c, mu, -1);
      load_spinor_df(ps, V, n, nb, mu == 0 && c[0] == 0 && bc_t < 0);
      load_link(U, V, mu, n, u);
      hop_accumulate(mu, false, u, nb, acc);
    }
  }
  cplx<dfl> d[12];
  load_spinor_df(ps, V, x, nb, false);
  clover_apply(clov, V, x, nb, d, dfl(0));
  cplx<double>* po = out + ro;
  const dfl half(0.5f);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    cplx<dfl> v = d[k] - half * acc[k];
    if (RESID) {
      const cplx<double> bb = bsrc[ro + (size_t)k * V + x];
      v = cmk<dfl>(df_from_double(bb.re), df_from_double(bb.im)) - v;
    }
    po[(size_t)k * V + x] = cmk<double>(df_to_double(v.re), df_to_double(v.im));
  }
}

// FP64 -> double-FP32 pairs rounded to nearest (operator data, converted once)
__global__ void k_double_to_df(dfl* __restrict__ dst, const double* __restrict__ src, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = src[i];
  const float hi = __double2float_rn(x);
  dst[i] = dfl(hi, __double2float_rn(__dsub_rn(x, (double)hi)));
}

// ---------------------------------------------------------------------------
// Segmented sum over groups of `seg` consecutive threads (seg a power of two);
// groups wider than a warp combine warp partials through shared memory.
template <typename T>
__device__ void seg_sum3(T& a, T& b, T& c, int seg, T* scratch) {
  const int w = seg < 32 ? seg : 32;
  for (int off = w >> 1; off >= 1; off >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, off);
    b += __shfl_xor_sync(0xffffffffu, b, off);
    c += __shfl_xor_sync(0xffffffffu, c, off);
  }
  if (seg > 32) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { scratch[3 * warp] = a; scratch[3 * warp + 1] = b; scratch[3 * warp + 2] = c; }
    __syncthreads();
    const int wps = seg >> 5;
    const int first = (warp / wps) * wps;
    a = b = c = T(0);
    for (int i = 0; i < wps; ++i) {
      a += scratch[3 * (first + i)];
      b += scratch[3 * (first + i) + 1];
      c += scratch[3 * (first + i) + 2];
    }
    __syncthreads();
  }
}

// One colour sweep of SAP on the fine level (multiplicative Schwarz, Sec. 1):
// for every SAP block B of the colour, rho_B = (b - D z)_B, k minimal-residual
// steps on D_B e = rho_B (hops leaving B dropped), then z_B += e_B.  Written in
// terms of z: the black sweep's rho = b - D z sees the red update, which is the
// same as r - D e with e the red correction.  One CTA segment of `seg` threads
// per block, one thread per site; the block's residual lives in shared memory.
template <typename T, typename LS, typename CS>
__global__ void k_fine_sap(cplx<T>* __restrict__ z, const cplx<T>* __restrict__ bsrc,
                           const LS* __restrict__ U, const CS* __restrict__ clov, Geom g, int bc_t,
                           size_t rstride, const int* __restrict__ blocks, int nblocks, int seg,
                           int k_mr, T shift) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* rs = reinterpret_cast<cplx<T>*>(smem_raw);            // [blockDim.x][12]
  T* scratch = reinterpret_cast<T*>(rs + (size_t)blockDim.x * 12);  // [warps][3]
  const int segs = blockDim.x / seg;
  const int s = threadIdx.x / seg;
  const int loc = threadIdx.x - s * seg;
  const int bi = blockIdx.x * segs + s;
  const bool active = (bi < nblocks) && (loc < g.vB);
  const int blk = active ? blocks[bi] : 0;
  const int x = blk * g.vB + loc;
  const int V = g.V;
  const size_t ro = (size_t)blockIdx.y * rstride;
  cplx<T>* pz = z + ro;
  int c[4] = {0, 0, 0, 0};
  cplx<T> r[12], xs[12], p[12], nb[12], u[9];
  if (active) {
    geom_coords(g, x, c);
    // rho = b - D z at x
    cplx<T> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = czero<T>();
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
      int n = geom_neighbor(g, c, mu, +1);
      T sgn = (mu == 0 && c[0] == g.L[0] - 1) ? T(bc_t) : T(1);
      load_spinor(pz, V, n, nb, sgn, -1);
      load_link(U, V, mu, x, u);
      hop_accumulate(mu, true, u, nb, acc);
      n = geom_neighbor(g, c, mu, -1);
      sgn = (mu == 0 && c[0] == 0) ? T(bc_t) : T(1);
      load_spinor(pz, V, n, nb, sgn, -1);
      load_link(U, V, mu, n, u);
      hop_accumulate(mu, false, u, nb, acc);
    }
    load_spinor(pz, V, x, nb, T(1), -1);
    clover_apply(clov, V, x, nb, p, shift);
    const cplx<T>* pb = bsrc + ro;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      r[k] = pb[(size_t)k * V + x] - (p[k] - T(0.5) * acc[k]);
      xs[k] = czero<T>();
    }
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) { r[k] = czero<T>(); xs[k] = czero<T>(); }
  }
  const int base = s * seg;   // shared-memory slot of the block's first site
#pragma unroll 1
  for (int it = 0; it < k_mr; ++it) {
#pragma unroll
    for (int k = 0; k < 12; ++k) rs[(size_t)threadIdx.x * 12 + k] = r[k];
    __syncthreads();
    T nre = T(0), nim = T(0), den = T(0);
    if (active) {
      cplx<T> acc[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = czero<T>();
#pragma unroll 1
      for (int mu = 0; mu < 4; ++mu) {
        // a block that spans the whole time extent keeps the wrapping hop, with its boundary sign
        if (hop_internal(g, c, mu, +1, g.B)) {
          const int n = geom_neighbor(g, c, mu, +1);
          const int sl = base + (n - blk * g.vB);
          const bool neg = mu == 0 && bc_t < 0 && c[0] == g.L[0] - 1;
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            const cplx<T> v = rs[(size_t)sl * 12 + k];
            nb[k] = cmk<T>(sign_flip(v.re, neg), sign_flip(v.im, neg));
          }
          load_link(U, V, mu, x, u);
          hop_accumulate(mu, true, u, nb, acc);
        }
        if (hop_internal(g, c, mu, -1, g.B)) {
          const int n = geom_neighbor(g, c, mu, -1);
          const int sl = base + (n - blk * g.vB);
          const bool neg = mu == 0 && bc_t < 0 && c[0] == 0;
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            const cplx<T> v = rs[(size_t)sl * 12 + k];
            nb[k] = cmk<T>(sign_flip(v.re, neg), sign_flip(v.im, neg));
          }
          load_link(U, V, mu, n, u);
          hop_accumulate(mu, false, u, nb, acc);
        }
      }
      clover_apply(clov, V, x, r, p, shift);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        p[k] = p[k] - T(0.5) * acc[k];
        const cplx<T> t = cdotc(p[k], r[k]);
        nre += t.re;
        nim += t.im;
        den += cnorm2(p[k]);
      }
    }
    seg_sum3(nre, nim, den, seg, scratch);
    const cplx<T> alpha = den > T(0) ? cmk<T>(nre / den, nim / den) : czero<T>();
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      cfma(xs[k], alpha, r[k]);
      r[k] = r[k] - alpha * p[k];
    }
    __syncthreads();
  }
  if (active) {
#pragma unroll
    for (int k = 0; k < 12; ++k) pz[(size_t)k * V + x] = pz[(size_t)k * V + x] + xs[k];
  }
}

// ---------------------------------------------------------------------------
// SAP colour sweep with the SAP block staged in shared memory by TMA.
//
// One CTA per SAP block (or several small blocks).  A single thread arms an
// mbarrier and issues 1-D bulk copies (cp.async.bulk, global -> shared) of the
// block's 36 link rows and its clover rows (72 reals, or 36 half2 pairs for
// FP16 storage), each a contiguous run of vB words in the component-major
// layout.  (4^4 blocks use the specialised kernel below.)  After the barrier completes,
// the k minimal-residual steps on D_B read links, clover and the residual only
// from shared memory; the neighbour slots inside the block are computed once.
// The CTA loops over the right-hand sides, so the operator is staged once per
// batch.  Waits are bounded: on a timeout the kernel records an error code,
// waits (bounded) for its copies and returns without touching z.
template <typename T, typename LS, typename CS>
__global__ void __launch_bounds__(256, 2) k_fine_sap_tma(cplx<T>* __restrict__ z, const cplx<T>* __restrict__ bsrc,
                                                      const LS* __restrict__ U, const CS* __restrict__ clov, Geom g,
                                                      int bc_t, size_t rstride, int nrhs, const int* __restrict__ blocks,
                                                      int nblocks, int seg, int k_mr, int* err, T shift) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int vB = g.vB;
  const int segs = blockDim.x / seg;
  constexpr int CR = 2 * ClovRows<CS>::per_chir;
  // per segment: links [36][vB] LS, clover [CR][vB] CS, residual [12][vB] cplx
  const size_t seg_bytes = (size_t)vB * (36 * sizeof(LS) + CR * sizeof(CS) + 12 * sizeof(cplx<T>));
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + (size_t)segs * seg_bytes);
  T* scratch = reinterpret_cast<T*>(bar + 2);
  const int s = threadIdx.x / seg;
  const int loc = threadIdx.x - s * seg;
  const int bi = blockIdx.x * segs + s;
  const bool active = (bi < nblocks) && (loc < vB);
  const int blk = (bi < nblocks) ? blocks[bi] : 0;
  unsigned char* sb = smem_raw + (size_t)s * seg_bytes;
  LS* Ls = reinterpret_cast<LS*>(sb);
  CS* Cs = reinterpret_cast<CS*>(Ls + 36 * vB);
  cplx<T>* Rs = reinterpret_cast<cplx<T>*>(Cs + CR * vB);
  const int V = g.V;
  // stage the operator of every segment's block
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x < 32) {
    int nseg = 0;
    for (int q = 0; q < segs; ++q) nseg += (blockIdx.x * segs + q < nblocks) ? 1 : 0;
    const unsigned bytes = (unsigned)(nseg * vB * (36 * sizeof(LS) + CR * sizeof(CS)));
    if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, bytes);
    __syncwarp();
    for (int q = 0; q < nseg; ++q) {
      const int bq = blocks[blockIdx.x * segs + q];
      unsigned char* sq = smem_raw + (size_t)q * seg_bytes;
      LS* Lq = reinterpret_cast<LS*>(sq);
      CS* Cq = reinterpret_cast<CS*>(Lq + 36 * vB);
      for (int cpy = threadIdx.x; cpy < 36 + CR; cpy += 32) {
        if (cpy < 36)
          bulk_g2s(Lq + (size_t)cpy * vB, U + (size_t)cpy * V + (size_t)bq * vB, (unsigned)(vB * sizeof(LS)), bar);
        else
          bulk_g2s(Cq + (size_t)(cpy - 36) * vB, clov + (size_t)(cpy - 36) * V + (size_t)bq * vB,
                   (unsigned)(vB * sizeof(CS)), bar);
      }
    }
  }
  // geometry of this thread's site (overlaps the copies)
  int l[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
  int nslot[8];
  T nsign[8];
  const int x = blk * vB + loc;
  if (active) {
    geom_coords(g, x, c);
    delin4(loc, g.B, l);
    const int st[4] = {g.B[1] * g.B[2] * g.B[3], g.B[2] * g.B[3], g.B[3], 1};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int mu = k >> 1, dir = (k & 1) ? -1 : +1;
      int nl = l[mu] + dir;
      bool internal = nl >= 0 && nl < g.B[mu];
      if (!internal && g.B[mu] == g.L[mu]) {
        internal = true;
        nl = (nl + g.B[mu]) % g.B[mu];
      }
      nslot[k] = internal ? loc + (nl - l[mu]) * st[mu] : -1;
      nsign[k] = (mu == 0 && ((dir > 0 && c[0] == g.L[0] - 1) || (dir < 0 && c[0] == 0))) ? T(bc_t) : T(1);
    }
  }
  const int ok = __syncthreads_and(mbar_wait_bounded(bar, 0) ? 1 : 0);
  if (!ok) {   // uniform across the CTA
    if (threadIdx.x == 0) atomicExch(err, 2);
    mbar_wait_bounded(bar, 0);
    return;
  }
  // The block residual lives only in shared memory (Rs); each thread keeps its
  // site's share of the correction e_B (xs) and of p = D_B r in registers.
  cplx<T> xs[12], p[12], nb[12], u[9];
  for (int rh = 0; rh < nrhs; ++rh) {
    cplx<T>* pz = z + (size_t)rh * rstride;
    if (active) {
      // rho = b - D z at x: hops to neighbours inside the block use the staged links
      cplx<T> acc[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = czero<T>();
#pragma unroll 1
      for (int k = 0; k < 8; ++k) {
        const int mu = k >> 1;
        const bool fwd = (k & 1) == 0;
        const int n = nslot[k] >= 0 ? blk * vB + nslot[k] : geom_neighbor(g, c, mu, fwd ? +1 : -1);
        load_spinor(pz, V, n, nb, nsign[k], -1);
        if (fwd) {
#pragma unroll
          for (int q = 0; q < 9; ++q) u[q] = ld_cplx(Ls, (size_t)(mu * 9 + q) * vB + loc);
        } else if (nslot[k] >= 0) {
#pragma unroll
          for (int q = 0; q < 9; ++q) u[q] = ld_cplx(Ls, (size_t)(mu * 9 + q) * vB + nslot[k]);
        } else {
          load_link(U, V, mu, n, u);
        }
        hop_accumulate(mu, fwd, u, nb, acc);
      }
      load_spinor(pz, V, x, nb, T(1), -1);
      clover_apply(Cs, vB, loc, nb, p, shift);
      const cplx<T>* pb = bsrc + (size_t)rh * rstride;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        Rs[(size_t)k * vB + loc] = pb[(size_t)k * V + x] - (p[k] - T(0.5) * acc[k]);
        xs[k] = czero<T>();
      }
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) xs[k] = czero<T>();
    }
    __syncthreads();
#pragma unroll 1
    for (int it = 0; it < k_mr; ++it) {
      T nre = T(0), nim = T(0), den = T(0);
      if (active) {
        cplx<T> acc[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = czero<T>();
#pragma unroll 1
        for (int k = 0; k < 8; ++k) {
          const int sl = nslot[k];
          if (sl < 0) continue;
          const int mu = k >> 1;
          const bool fwd = (k & 1) == 0;
          const bool neg = nsign[k] < T(0);
#pragma unroll
          for (int q = 0; q < 12; ++q) {
            const cplx<T> v = Rs[(size_t)q * vB + sl];
            nb[q] = cmk<T>(sign_flip(v.re, neg), sign_flip(v.im, neg));
          }
          const int ls = fwd ? loc : sl;
#pragma unroll
          for (int q = 0; q < 9; ++q) u[q] = ld_cplx(Ls, (size_t)(mu * 9 + q) * vB + ls);
          hop_accumulate(mu, fwd, u, nb, acc);
        }
#pragma unroll
        for (int q = 0; q < 12; ++q) nb[q] = Rs[(size_t)q * vB + loc];   // own residual
        clover_apply(Cs, vB, loc, nb, p, shift);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          p[k] = p[k] - T(0.5) * acc[k];
          const cplx<T> t = cdotc(p[k], nb[k]);
          nre += t.re;
          nim += t.im;
          den += cnorm2(p[k]);
        }
      }
      seg_sum3(nre, nim, den, seg, scratch);
      const cplx<T> alpha = den > T(0) ? cmk<T>(nre / den, nim / den) : czero<T>();
      __syncthreads();   // every read of Rs for p is done before Rs changes
      if (active) {
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          const cplx<T> r = Rs[(size_t)k * vB + loc];
          cfma(xs[k], alpha, r);
          Rs[(size_t)k * vB + loc] = r - alpha * p[k];
        }
      }
      __syncthreads();
    }
    if (active) {
#pragma unroll
      for (int k = 0; k < 12; ++k) pz[(size_t)k * V + x] = pz[(size_t)k * V + x] + xs[k];
    }
  }
}

// ---------------------------------------------------------------------------
// SAP colour sweep for 4^4 blocks (the SAP block of the paper's fine level,
// Table 1): one CTA of 256 threads per block, one thread per site.  The block
// volume is a compile-time constant, so every shared-memory address below is
// a thread base plus an immediate, and the eight hop directions are unrolled
// with the spin projection of each direction fixed at compile time.
//
// Staging (cp.async.bulk on two mbarriers): the block's 36 link rows and its
// clover rows (bar[0], once), and the block's own 12 rows of z (bar[1], once
// per right-hand side) into the residual buffer Rs.  rho = b - D z then reads
// internal neighbours from Rs and only the hops leaving the block from global
// memory.  Each minimal-residual step takes two barriers: one after the warp
// partials of <p, r> and |p|^2 are written (every read of Rs for p is done
// by then), one after r is updated.  The partials are summed over the eight
// warps in a fixed order by every thread, so all threads get the same alpha.
// Waits are bounded: on a timeout the kernel sets *err, waits (bounded) for its
// copies and returns without touching z.
template <typename LS, typename CS>
__global__ void __launch_bounds__(256, 2) k_fine_sap_b4(cplx<float>* __restrict__ z,
                                                     const cplx<float>* __restrict__ bsrc, const LS* __restrict__ U,
                                                     const CS* __restrict__ clov, Geom g, int bc_t, size_t rstride,
                                                     int nrhs, const int* __restrict__ blocks, int k_mr, int* err,
                                                     float shift) {
  using C = cplx<float>;
  constexpr int VB = 256;
  constexpr int CR = 2 * ClovRows<CS>::per_chir;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LS* Ls = reinterpret_cast<LS*>(smem_raw);                       // [36][VB]
  CS* Cs = reinterpret_cast<CS*>(Ls + 36 * VB);                   // [CR][VB]
  C* Rs = reinterpret_cast<C*>(Cs + CR * VB);                     // [12][VB]: z of the block, then r
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(Rs + 12 * VB);
  float* scratch = reinterpret_cast<float*>(bar + 2);             // [2][8 warps][3]
  const int loc = threadIdx.x, lane = loc & 31, warp = loc >> 5;
  // the next sweep (launched with programmatic stream serialization) may start staging its
  // links and clover term while this one runs; it waits for this grid before reading z or b
  pdl_launch_dependents();
  const int blk = blocks[blockIdx.x];
  const int V = g.V;
  const int x = blk * VB + loc;
  if (loc == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
  }
  __syncthreads();
  if (warp == 0) {   // links and clover term: never written by the kernels this launch may overlap
    if (lane == 0) {
      mbar_arrive_expect_tx(&bar[0], (unsigned)(VB * (36 * sizeof(LS) + CR * sizeof(CS))));
      mbar_arrive_expect_tx(&bar[1], (unsigned)(12 * VB * sizeof(C)));
    }
    __syncwarp();
    for (int cpy = lane; cpy < 36 + CR; cpy += 32) {
      if (cpy < 36)
        bulk_g2s(Ls + (size_t)cpy * VB, U + (size_t)cpy * V + (size_t)blk * VB, VB * sizeof(LS), &bar[0]);
      else
        bulk_g2s(Cs + (size_t)(cpy - 36) * VB, clov + (size_t)(cpy - 36) * V + (size_t)blk * VB, VB * sizeof(CS),
                 &bar[0]);
    }
  }
  pdl_wait();   // the previous kernel's z and b are complete from here on
  if (warp == 0 && lane < 12)
    bulk_g2s(Rs + (size_t)lane * VB, z + (size_t)lane * V + (size_t)blk * VB, VB * sizeof(C), &bar[1]);
  // site geometry (overlaps the copies): local coordinates l_mu = (loc / st_mu) % 4,
  // st = (64, 16, 4, 1); a hop is internal if it stays in the block, or wraps
  // around a lattice direction of extent 4 that the block spans
  int c[4];
  geom_coords(g, x, c);
  unsigned inmask = 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int l = (loc >> (6 - 2 * mu)) & 3;
    const bool wrap = g.L[mu] == 4;
    if (l < 3 || wrap) inmask |= 1u << (2 * mu);
    if (l > 0 || wrap) inmask |= 1u << (2 * mu + 1);
  }
  const bool neg_tf = bc_t < 0 && c[0] == g.L[0] - 1;   // forward time hop wraps the lattice
  const bool neg_tb = bc_t < 0 && c[0] == 0;            // backward time hop wraps the lattice
  auto slot = [&](int mu, bool fwd) {
    const int st = 1 << (6 - 2 * mu);
    const int l = (loc >> (6 - 2 * mu)) & 3;
    return fwd ? (l < 3 ? loc + st : loc - 3 * st) : (l > 0 ? loc - st : loc + 3 * st);
  };
  bool ok = __syncthreads_and(mbar_wait_bounded(&bar[0], 0) ? 1 : 0);
  C xs[12], p[12], nb[12], u[9];
  int zphase = 0;   // phase of the last z copy issued on bar[1]
  for (int rh = 0; rh < nrhs && ok; ++rh) {
    C* pz = z + (size_t)rh * rstride;
    zphase = rh & 1;
    if (rh > 0 && warp == 0) {   // every access of Rs for the previous right-hand side is done (last barrier)
      fence_proxy_async_shared();
      if (lane == 0) mbar_arrive_expect_tx(&bar[1], (unsigned)(12 * VB * sizeof(C)));
      __syncwarp();
      if (lane < 12) bulk_g2s(Rs + (size_t)lane * VB, pz + (size_t)lane * V + (size_t)blk * VB, VB * sizeof(C), &bar[1]);
    }
    ok = __syncthreads_and(mbar_wait_bounded(&bar[1], zphase) ? 1 : 0);
    if (!ok) break;
    // rho = b - D z at x
    {
      C acc[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = czero<float>();
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int mu = k >> 1;
        const bool fwd = (k & 1) == 0;
        const bool neg = mu == 0 && (fwd ? neg_tf : neg_tb);
        if (inmask & (1u << k)) {
          const int sl = slot(mu, fwd);
#pragma unroll
          for (int q = 0; q < 12; ++q) {
            const C v = Rs[q * VB + sl];
            nb[q] = cmk<float>(sign_flip(v.re, neg), sign_flip(v.im, neg));
          }
          const int ls = fwd ? loc : sl;
#pragma unroll
          for (int q = 0; q < 9; ++q) u[q] = ld_cplx(Ls, (size_t)((mu * 9 + q) * VB + ls));
        } else {
          const int n = geom_neighbor(g, c, mu, fwd ? +1 : -1);
          load_spinor(pz, V, n, nb, neg ? -1.f : 1.f, -1);
          if (fwd) {
#pragma unroll
            for (int q = 0; q < 9; ++q) u[q] = ld_cplx(Ls, (size_t)((mu * 9 + q) * VB + loc));
          } else {
            load_link(U, V, mu, n, u);
          }
        }
        hop_accumulate(mu, fwd, u, nb, acc);
      }
#pragma unroll
      for (int q = 0; q < 12; ++q) nb[q] = Rs[q * VB + loc];
      clover_apply(Cs, VB, loc, nb, p, shift);
      const C* pb = bsrc + (size_t)rh * rstride;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        nb[k] = pb[(size_t)k * V + x] - (p[k] - 0.5f * acc[k]);
        xs[k] = czero<float>();
      }
    }
    __syncthreads();   // every read of the staged z is done
#pragma unroll
    for (int k = 0; k < 12; ++k) Rs[k * VB + loc] = nb[k];
    __syncthreads();
#pragma unroll 1
    for (int it = 0; it < k_mr; ++it) {
      C acc[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = czero<float>();
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int mu = k >> 1;
        const bool fwd = (k & 1) == 0;
        if (inmask & (1u << k)) {
          const bool neg = mu == 0 && (fwd ? neg_tf : neg_tb);
          const int sl = slot(mu, fwd);
#pragma unroll
          for (int q = 0; q < 12; ++q) {
            const C v = Rs[q * VB + sl];
            nb[q] = cmk<float>(sign_flip(v.re, neg), sign_flip(v.im, neg));
          }
          const int ls = fwd ? loc : sl;
#pragma unroll
          for (int q = 0; q < 9; ++q) u[q] = ld_cplx(Ls, (size_t)((mu * 9 + q) * VB + ls));
          hop_accumulate(mu, fwd, u, nb, acc);
        }
      }
#pragma unroll
      for (int q = 0; q < 12; ++q) nb[q] = Rs[q * VB + loc];   // own residual, kept for the update
      clover_apply(Cs, VB, loc, nb, p, shift);
      float nre = 0.f, nim = 0.f, den = 0.f;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        p[k] = p[k] - 0.5f * acc[k];
        cdotc_acc(nre, nim, p[k], nb[k]);
        cnorm2_acc(den, p[k]);
      }
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
        nre += __shfl_xor_sync(0xffffffffu, nre, off);
        nim += __shfl_xor_sync(0xffffffffu, nim, off);
        den += __shfl_xor_sync(0xffffffffu, den, off);
      }
      float* sc = scratch + (it & 1) * 24;
      if (lane == 0) {
        sc[3 * warp] = nre;
        sc[3 * warp + 1] = nim;
        sc[3 * warp + 2] = den;
      }
      __syncthreads();
      nre = nim = den = 0.f;
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        nre += sc[3 * w];
        nim += sc[3 * w + 1];
        den += sc[3 * w + 2];
      }
      const C alpha = den > 0.f ? cmk<float>(nre / den, nim / den) : czero<float>();
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        cfma(xs[k], alpha, nb[k]);
        Rs[k * VB + loc] = nb[k] - alpha * p[k];
      }
      __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) pz[(size_t)k * V + x] = pz[(size_t)k * V + x] + xs[k];
  }
  if (!ok) {   // uniform across the CTA
    if (loc == 0) atomicExch(err, 2);
    mbar_wait_bounded(&bar[0], 0);
    mbar_wait_bounded(&bar[1], zphase);
  }
}

// ---------------------------------------------------------------------------
// Clover construction (FP64).  Q_mu_nu(x) = sum of the four plaquette leaves
// at x in the mu-nu plane; A(x) = (m0 + 4) - (c_sw / 16) sum_{mu<nu}
// (gamma_mu gamma_nu) (x) (Q_mu_nu - Q_mu_nu^+), which is the sum over ordered
// pairs with weight -(c_sw/32).  Stored as two packed Hermitian 6x6 blocks.
__constant__ double2 c_gg[6][4][4];   // gamma_mu gamma_nu for the 6 planes mu < nu

using cd = cplx<double>;

DD_HD void m3_mul(const cd* a, const cd* b, cd* c) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cd s = a[i * 3] * b[j];
      cfma(s, a[i * 3 + 1], b[3 + j]);
      cfma(s, a[i * 3 + 2], b[6 + j]);
      c[i * 3 + j] = s;
    }
}
DD_HD void m3_dag(const cd* a, cd* c) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c[i * 3 + j] = cconj(a[j * 3 + i]);
}

__device__ void lex_link(const cd* __restrict__ gl, const int L[4], const int c[4], int dshift0, int s0,
                         int dshift1, int s1, int mu, cd* out) {
  int n[4] = {c[0], c[1], c[2], c[3]};
  if (s0) { n[dshift0] = (n[dshift0] + s0 + L[dshift0]) % L[dshift0]; }
  if (s1) { n[dshift1] = (n[dshift1] + s1 + L[dshift1]) % L[dshift1]; }
  const size_t site = (size_t)lin4(n, L);
  for (int k = 0; k < 9; ++k) out[k] = gl[(site * 4 + mu) * 9 + k];
}

__global__ void k_clover_build(double* __restrict__ clov, const cd* __restrict__ gl, Geom g, double m0,
                               double csw) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.V) return;
  int c[4];
  geom_coords(g, x, c);
  cd A[2][6][6];
  for (int ch = 0; ch < 2; ++ch)
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) A[ch][i][j] = cmk(i == j ? m0 + 4.0 : 0.0, 0.0);
  if (csw != 0.0) {
    int plane = 0;
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu, ++plane) {
        cd Q[9], t1[9], t2[9], a[9], b[9], cc[9], d[9], da[9];
        for (int k = 0; k < 9; ++k) Q[k] = czero<double>();
        // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
        lex_link(gl, g.L, c, 0, 0, 0, 0, mu, a);
        lex_link(gl, g.L, c, mu, 1, 0, 0, nu, b);
        lex_link(gl, g.L, c, nu, 1, 0, 0, mu, cc);
        lex_link(gl, g.L, c, 0, 0, 0, 0, nu, d);
        m3_mul(a, b, t1); m3_dag(cc, da); m3_mul(t1, da, t2); m3_dag(d, da); m3_mul(t2, da, t1);
        for (int k = 0; k < 9; ++k) Q[k] = Q[k] + t1[k];
        // leaf 2: U_nu(x) U_mu(x+nu-mu)^+ U_nu(x-mu)^+ U_mu(x-mu)
        lex_link(gl, g.L, c, 0, 0, 0, 0, nu, a);
        lex_link(gl, g.L, c, nu, 1, mu, -1, mu, b);
        lex_link(gl, g.L, c, mu, -1, 0, 0, nu, cc);
        lex_link(gl, g.L, c, mu, -1, 0, 0, mu, d);
        m3_dag(b, da); m3_mul(a, da, t1); m3_dag(cc, da); m3_mul(t1, da, t2); m3_mul(t2, d, t1);
        for (int k = 0; k < 9; ++k) Q[k] = Q[k] + t1[k];
        // leaf 3: U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu)
        lex_link(gl, g.L, c, mu, -1, 0, 0, mu, a);
        lex_link(gl, g.L, c, mu, -1, nu, -1, nu, b);
        lex_link(gl, g.L, c, mu, -1, nu, -1, mu, cc);
        lex_link(gl, g.L, c, nu, -1, 0, 0, nu, d);
        m3_dag(a, da); m3_dag(b, t2); m3_mul(da, t2, t1); m3_mul(t1, cc, t2); m3_mul(t2, d, t1);
        for (int k = 0; k < 9; ++k) Q[k] = Q[k] + t1[k];
        // leaf 4: U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^+
        lex_link(gl, g.L, c, nu, -1, 0, 0, nu, a);
        lex_link(gl, g.L, c, nu, -1, 0, 0, mu, b);
        lex_link(gl, g.L, c, nu, -1, mu, 1, nu, cc);
        lex_link(gl, g.L, c, 0, 0, 0, 0, mu, d);
        m3_dag(a, da); m3_mul(da, b, t1); m3_mul(t1, cc, t2); m3_dag(d, da); m3_mul(t2, da, t1);
        for (int k = 0; k < 9; ++k) Q[k] = Q[k] + t1[k];
        cd F[9];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) F[i * 3 + j] = Q[i * 3 + j] - cconj(Q[j * 3 + i]);
        const double w = -csw / 16.0;
        for (int ch = 0; ch < 2; ++ch)
          for (int s = 0; s < 2; ++s)
            for (int t = 0; t < 2; ++t) {
              const double2 gv = c_gg[plane][2 * ch + s][2 * ch + t];
              const cd gs = cmk(w * gv.x, w * gv.y);
              for (int a3 = 0; a3 < 3; ++a3)
                for (int b3 = 0; b3 < 3; ++b3) cfma(A[ch][s * 3 + a3][t * 3 + b3], gs, F[a3 * 3 + b3]);
            }
      }
  }
  for (int ch = 0; ch < 2; ++ch) {
    double* o = clov + (size_t)ch * 36 * g.V + x;
    for (int i = 0; i < 6; ++i) o[(size_t)i * g.V] = A[ch][i][i].re;
    for (int i = 0; i < 6; ++i)
      for (int j = i + 1; j < 6; ++j) {
        const int p = 6 + 2 * herm_off(i, j);
        o[(size_t)p * g.V] = A[ch][i][j].re;
        o[(size_t)(p + 1) * g.V] = A[ch][i][j].im;
      }
  }
}

// ---------------------------------------------------------------------------
// Inverse of the site-diagonal part A(x) = (m0 + 4) + C(x) on the fine level: per site and
// chirality a Hermitian 6x6 block, factored A = L D L^+ (L unit lower triangular, D real) in
// FP64 and inverted column by column (forward and back substitution).  Output in the packed
// Hermitian layout of the clover term.  A vanishing or non-finite pivot sets *err.
__global__ void k_clover_inverse(double* __restrict__ inv, const double* __restrict__ clov, int V, int* err) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)2 * V) return;
  const int ch = (int)(t / V), x = (int)(t - (size_t)ch * V);
  const double* a = clov + (size_t)ch * 36 * V + x;
  cd A[6][6];
  for (int i = 0; i < 6; ++i) A[i][i] = cmk(a[(size_t)i * V], 0.0);
  for (int i = 0; i < 6; ++i)
    for (int j = i + 1; j < 6; ++j) {
      const int p = 6 + 2 * herm_off(i, j);
      A[i][j] = cmk(a[(size_t)p * V], a[(size_t)(p + 1) * V]);
      A[j][i] = cconj(A[i][j]);
    }
  // L D L^+ : column j of L below the diagonal and D_j
  cd L[6][6];
  double Dg[6];
  for (int j = 0; j < 6; ++j) {
    double d = A[j][j].re;
    for (int k = 0; k < j; ++k) d -= Dg[k] * cnorm2(L[j][k]);
    if (!(fabs(d) > 1e-300) || !isfinite(d)) {
      atomicExch(err, 1);
      return;
    }
    Dg[j] = d;
    for (int i = j + 1; i < 6; ++i) {
      cd s = A[i][j];
      for (int k = 0; k < j; ++k) s = s - Dg[k] * (L[i][k] * cconj(L[j][k]));
      L[i][j] = (1.0 / d) * s;
    }
  }
  // X = A^{-1}: solve L y = e_c, then D, then L^+ x = y, for each column c
  cd X[6][6];
  for (int c = 0; c < 6; ++c) {
    cd y[6];
    for (int i = 0; i < 6; ++i) {
      cd s = cmk(i == c ? 1.0 : 0.0, 0.0);
      for (int k = 0; k < i; ++k) s = s - L[i][k] * y[k];
      y[i] = s;
    }
    for (int i = 0; i < 6; ++i) y[i] = (1.0 / Dg[i]) * y[i];
    for (int i = 5; i >= 0; --i) {
      cd s = y[i];
      for (int k = i + 1; k < 6; ++k) s = s - cconj(L[k][i]) * X[k][c];
      X[i][c] = s;
    }
  }
  double* o = inv + (size_t)ch * 36 * V + x;
  for (int i = 0; i < 6; ++i) o[(size_t)i * V] = X[i][i].re;
  for (int i = 0; i < 6; ++i)
    for (int j = i + 1; j < 6; ++j) {
      const int p = 6 + 2 * herm_off(i, j);
      o[(size_t)p * V] = X[i][j].re;
      o[(size_t)(p + 1) * V] = X[i][j].im;
    }
}

// Per-site tables read by the Schur SAP kernel: the clover term on even sites, the inverse of
// A(x) on odd sites.  FP32: [2][36][V] reals (even sites with the (m0 + 4) shift, as the FP32
// clover); FP16: [2][18][V] pairs of reals (even sites without the shift, as the FP16 clover).
__global__ void k_clover_mix32(float* __restrict__ mix, const double* __restrict__ clov,
                               const double* __restrict__ inv, Geom g) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)72 * g.V) return;
  const int x = (int)(i % g.V);
  int c[4];
  geom_coords(g, x, c);
  mix[i] = (float)(geom_parity(c) ? inv[i] : clov[i]);
}

__global__ void k_clover_mix_half(__half2* __restrict__ mix, const double* __restrict__ clov,
                                  const double* __restrict__ inv, Geom g, double shift) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)36 * g.V) return;
  const int row = (int)(i / g.V), x = (int)(i - (size_t)row * g.V);
  const int ch = row / 18, p = 2 * (row - 18 * ch);
  int c[4];
  geom_coords(g, x, c);
  const bool odd = geom_parity(c) != 0;
  const double* src = odd ? inv : clov;
  const double sh = odd ? 0.0 : shift;
  const double a0 = src[(size_t)(ch * 36 + p) * g.V + x], a1 = src[(size_t)(ch * 36 + p + 1) * g.V + x];
  mix[i] = __halves2half2(__double2half(p < 6 ? a0 - sh : a0), __double2half(p + 1 < 6 ? a1 - sh : a1));
}

// ---------------------------------------------------------------------------
// SAP colour sweep for 4^4 blocks with each block solved on its even-odd Schur complement
// (the block solve of the oracle's schur reading): with D = A - H/2 (A the site-diagonal part,
// H the hop sum) and H^B the hops that stay inside the block,
//   t_o   = A_o^{-1} rho_o = A_o^{-1} (b_o + H z / 2) - z_o
//   r_e   = rhohat_e = rho_e + H^B t_o / 2
//   k MR steps on  Dhat r = A_e r - H^B A_o^{-1} H^B r / 4   (alpha per block over even sites)
//   x_o   = t_o + A_o^{-1} H^B x_e / 2
// so no step needs A on odd sites: the staged per-site table holds A's clover term on even
// sites and A^{-1} on odd sites.  One CTA of 128 threads per block; thread t owns the two
// x-neighbours 2t, 2t+1 of the block (one even, one odd site), so every warp works on one parity
// at a time.  Staging and bounded waits as in the kernel above; the residual buffer Rs holds z,
// then r on even and the odd-site temporaries on odd sites; Ts holds t_o.
template <typename LS, typename CS>
__global__ void __launch_bounds__(128, 2) k_fine_sap_b4_eo(cplx<float>* __restrict__ z,
                                                        const cplx<float>* __restrict__ bsrc,
                                                        const LS* __restrict__ U, const CS* __restrict__ mix,
                                                        Geom g, int bc_t, size_t rstride, int nrhs,
                                                        const int* __restrict__ blocks, int k_mr, int* err,
                                                        float shift) {
  using C = cplx<float>;
  constexpr int VB = 256;
  constexpr int CR = 2 * ClovRows<CS>::per_chir;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LS* Ls = reinterpret_cast<LS*>(smem_raw);                       // [36][VB]
  CS* Cs = reinterpret_cast<CS*>(Ls + 36 * VB);                   // [CR][VB]
  C* Rs = reinterpret_cast<C*>(Cs + CR * VB);                     // [12][VB]
  C* Ts = Rs + 12 * VB;                                           // [12][128]: t_o of thread t
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(Ts + 12 * 128);
  float* scratch = reinterpret_cast<float*>(bar + 2);             // [2][4 warps][3]
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int blk = blocks[blockIdx.x];
  const int V = g.V;
  const int la = 2 * t;
  const int pa = (((la >> 6) & 3) + ((la >> 4) & 3) + ((la >> 2) & 3)) & 1;   // la & 3 is 0 or 2
  const int le = la + pa, lo = la + 1 - pa;                                     // even, odd site
  const int xe = blk * VB + le, xo = blk * VB + lo;
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
  }
  __syncthreads();
  if (warp == 0) {
    if (lane == 0) {
      mbar_arrive_expect_tx(&bar[0], (unsigned)(VB * (36 * sizeof(LS) + CR * sizeof(CS))));
      mbar_arrive_expect_tx(&bar[1], (unsigned)(12 * VB * sizeof(C)));
    }
    __syncwarp();
    for (int cpy = lane; cpy < 36 + CR + 12; cpy += 32) {
      if (cpy < 36)
        bulk_g2s(Ls + (size_t)cpy * VB, U + (size_t)cpy * V + (size_t)blk * VB, VB * sizeof(LS), &bar[0]);
      else if (cpy < 36 + CR)
        bulk_g2s(Cs + (size_t)(cpy - 36) * VB, mix + (size_t)(cpy - 36) * V + (size_t)blk * VB, VB * sizeof(CS),
                 &bar[0]);
      else
        bulk_g2s(Rs + (size_t)(cpy - 36 - CR) * VB, z + (size_t)(cpy - 36 - CR) * V + (size_t)blk * VB,
                 VB * sizeof(C), &bar[1]);
    }
  }
  // geometry of the two sites: internal-hop masks and the time-boundary signs
  int ce[4], co[4];
  geom_coords(g, xe, ce);
  geom_coords(g, xo, co);
  auto inmask_of = [&](int l) {
    unsigned m = 0;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int q = (l >> (6 - 2 * mu)) & 3;
      const bool wrap = g.L[mu] == 4;
      if (q < 3 || wrap) m |= 1u << (2 * mu);
      if (q > 0 || wrap) m |= 1u << (2 * mu + 1);
    }
    return m;
  };
  const unsigned im_e = inmask_of(le), im_o = inmask_of(lo);
  const bool ntf_e = bc_t < 0 && ce[0] == g.L[0] - 1, ntb_e = bc_t < 0 && ce[0] == 0;
  const bool ntf_o = bc_t < 0 && co[0] == g.L[0] - 1, ntb_o = bc_t < 0 && co[0] == 0;
  auto slot = [](int l, int mu, bool fwd) {
    const int st = 1 << (6 - 2 * mu);
    const int q = (l >> (6 - 2 * mu)) & 3;
    return fwd ? (q < 3 ? l + st : l - 3 * st) : (q > 0 ? l - st : l + 3 * st);
  };
  C nb[12], u[9];
  // acc = sum of the hops of site l (at x, coordinates c) that stay in the block, from Rs
  auto hops_in = [&](int l, unsigned inm, bool ntf, bool ntb, C acc[12]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = czero<float>();
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int mu = k >> 1;
      const bool fwd = (k & 1) == 0;
      if (inm & (1u << k)) {
        const bool neg = mu == 0 && (fwd ? ntf : ntb);
        const int sl = slot(l, mu, fwd);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
          const C v = Rs[q * VB + sl];
          nb[q] = cmk<float>(sign_flip(v.re, neg), sign_flip(v.im, neg));
        }
        const int ls = fwd ? l : sl;
#pragma unroll
        for (int q = 0; q < 9; ++q) u[q] = ld_cplx(Ls, (size_t)((mu * 9 + q) * VB + ls));
        hop_accumulate(mu, fwd, u, nb, acc);
      }
    }
  };
  // acc = H z at site l: internal hops from Rs, the others from global z and links
  auto hops_all = [&](const C* pz, int l, int x, const int* c, unsigned inm, bool ntf, bool ntb, C acc[12]) {
    hops_in(l, inm, ntf, ntb, acc);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int mu = k >> 1;
      const bool fwd = (k & 1) == 0;
      if (!(inm & (1u << k))) {
        const bool neg = mu == 0 && (fwd ? ntf : ntb);
        const int n = geom_neighbor(g, c, mu, fwd ? +1 : -1);
        load_spinor(pz, V, n, nb, neg ? -1.f : 1.f, -1);
        if (fwd) {
#pragma unroll
          for (int q = 0; q < 9; ++q) u[q] = ld_cplx(Ls, (size_t)((mu * 9 + q) * VB + l));
        } else {
          load_link(U, V, mu, n, u);
        }
        hop_accumulate(mu, fwd, u, nb, acc);
      }
    }
  };
  bool ok = __syncthreads_and(mbar_wait_bounded(&bar[0], 0) ? 1 : 0);
  C re[12], xe_[12], p[12], acc[12];
  int zphase = 0;
  for (int rh = 0; rh < nrhs && ok; ++rh) {
    C* pz = z + (size_t)rh * rstride;
    const C* pb = bsrc + (size_t)rh * rstride;
    zphase = rh & 1;
    if (rh > 0 && warp == 0) {   // every access of Rs for the previous right-hand side is done
      fence_proxy_async_shared();
      if (lane == 0) mbar_arrive_expect_tx(&bar[1], (unsigned)(12 * VB * sizeof(C)));
      __syncwarp();
      if (lane < 12) bulk_g2s(Rs + (size_t)lane * VB, pz + (size_t)lane * V + (size_t)blk * VB, VB * sizeof(C), &bar[1]);
    }
    ok = __syncthreads_and(mbar_wait_bounded(&bar[1], zphase) ? 1 : 0);
    if (!ok) break;
    // rho_e = b_e - A_e z_e + H z / 2 (even site); t_o = A_o^{-1} (b_o + H z / 2) - z_o (odd site)
    hops_all(pz, le, xe, ce, im_e, ntf_e, ntb_e, acc);
#pragma unroll
    for (int q = 0; q < 12; ++q) nb[q] = Rs[q * VB + le];
    clover_apply(Cs, VB, le, nb, p, shift);
#pragma unroll
    for (int k = 0; k < 12; ++k) re[k] = pb[(size_t)k * V + xe] - (p[k] - 0.5f * acc[k]);
    hops_all(pz, lo, xo, co, im_o, ntf_o, ntb_o, acc);
#pragma unroll
    for (int k = 0; k < 12; ++k) nb[k] = pb[(size_t)k * V + xo] + 0.5f * acc[k];
    clover_apply(Cs, VB, lo, nb, p, 0.f);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      p[k] = p[k] - Rs[k * VB + lo];
      Ts[k * 128 + t] = p[k];
    }
    __syncthreads();   // every read of the staged z is done
#pragma unroll
    for (int k = 0; k < 12; ++k) Rs[k * VB + lo] = p[k];
    __syncthreads();
    // r_e = rhohat_e = rho_e + H^B t_o / 2
    hops_in(le, im_e, ntf_e, ntb_e, acc);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      re[k] = re[k] + 0.5f * acc[k];
      xe_[k] = czero<float>();
      Rs[k * VB + le] = re[k];
    }
    __syncthreads();
#pragma unroll 1
    for (int it = 0; it < k_mr; ++it) {
      // odd stage: s_o = A_o^{-1} H^B r
      hops_in(lo, im_o, ntf_o, ntb_o, acc);
      clover_apply(Cs, VB, lo, acc, p, 0.f);
#pragma unroll
      for (int k = 0; k < 12; ++k) Rs[k * VB + lo] = p[k];
      __syncthreads();
      // even stage: p = A_e r - H^B s_o / 4
      hops_in(le, im_e, ntf_e, ntb_e, acc);
      clover_apply(Cs, VB, le, re, p, shift);
      float nre = 0.f, nim = 0.f, den = 0.f;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        p[k] = p[k] - 0.25f * acc[k];
        cdotc_acc(nre, nim, p[k], re[k]);
        cnorm2_acc(den, p[k]);
      }
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
        nre += __shfl_xor_sync(0xffffffffu, nre, off);
        nim += __shfl_xor_sync(0xffffffffu, nim, off);
        den += __shfl_xor_sync(0xffffffffu, den, off);
      }
      float* sc = scratch + (it & 1) * 12;
      if (lane == 0) {
        sc[3 * warp] = nre;
        sc[3 * warp + 1] = nim;
        sc[3 * warp + 2] = den;
      }
      __syncthreads();
      nre = nim = den = 0.f;
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        nre += sc[3 * w];
        nim += sc[3 * w + 1];
        den += sc[3 * w + 2];
      }
      const C alpha = den > 0.f ? cmk<float>(nre / den, nim / den) : czero<float>();
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        cfma(xe_[k], alpha, re[k]);
        re[k] = re[k] - alpha * p[k];
        Rs[k * VB + le] = re[k];
      }
      __syncthreads();
    }
    // x_o = t_o + A_o^{-1} H^B x_e / 2;  z += x
#pragma unroll
    for (int k = 0; k < 12; ++k) Rs[k * VB + le] = xe_[k];
    __syncthreads();
    hops_in(lo, im_o, ntf_o, ntb_o, acc);
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = 0.5f * acc[k];
    clover_apply(Cs, VB, lo, acc, p, 0.f);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      pz[(size_t)k * V + xo] = pz[(size_t)k * V + xo] + (Ts[k * 128 + t] + p[k]);
      pz[(size_t)k * V + xe] = pz[(size_t)k * V + xe] + xe_[k];
    }
    __syncthreads();   // Rs is read no more before the next right-hand side's copy
  }
  if (!ok) {   // uniform across the CTA
    if (t == 0) atomicExch(err, 2);
    mbar_wait_bounded(&bar[0], 0);
    mbar_wait_bounded(&bar[1], zphase);
  }
}

// gauge field from the ABI layout [lex site][mu][3][3] (FP64) to [mu][9][V]
template <typename T>
__global__ void k_links_import(cplx<T>* __restrict__ U, const cd* __restrict__ gl, Geom g) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.V) return;
  int c[4];
  geom_coords(g, x, c);
  const size_t site = (size_t)lin4(c, g.L);
  for (int mu = 0; mu < 4; ++mu)
    for (int k = 0; k < 9; ++k) U[(size_t)(mu * 9 + k) * g.V + x] = ccast<T>(gl[(site * 4 + mu) * 9 + k]);
}

// fine fields between the ABI layout [n][lex site][12] (FP64) and [n][12][V] of T
template <typename T>
__global__ void k_fine_import(cplx<T>* __restrict__ dst, const cd* __restrict__ src, Geom g, size_t rstride) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.V) return;
  int c[4];
  geom_coords(g, x, c);
  const size_t site = (size_t)lin4(c, g.L);
  const cd* s = src + (size_t)blockIdx.y * g.V * 12 + site * 12;
  cplx<T>* d = dst + (size_t)blockIdx.y * rstride;
  for (int k = 0; k < 12; ++k) d[(size_t)k * g.V + x] = ccast<T>(s[k]);
}

template <typename T>
__global__ void k_fine_export(cd* __restrict__ dst, const cplx<T>* __restrict__ src, Geom g, size_t rstride) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.V) return;
  int c[4];
  geom_coords(g, x, c);
  const size_t site = (size_t)lin4(c, g.L);
  cd* d = dst + (size_t)blockIdx.y * g.V * 12 + site * 12;
  const cplx<T>* s = src + (size_t)blockIdx.y * rstride;
  for (int k = 0; k < 12; ++k) d[k] = ccast<double>(s[(size_t)k * g.V + x]);
}

// ---------------------------------------------------------------------------
// Allocation-free residual norms ||b - D x|| / ||b|| for callers that cannot
// allocate device memory.  The reduction partials live in a file-scope device
// array instead of a cudaMalloc'ed scratch buffer; b and x are read in the ABI
// layout directly, so no conversion buffer is needed either.  The residual at a
// site is computed with the same device functions and the same order of
// operations as k_fine_dslash, so it is bit-identical to the library's own
// residual; only the order of the final sums differs.
constexpr int NOALLOC_MAX_RHS = 64;
constexpr int NOALLOC_CHUNKS = 1024;
__device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_RHS * NOALLOC_CHUNKS * 2];
__device__ __align__(256) double g_noalloc_out[NOALLOC_MAX_RHS];

__global__ void k_resnorm_partials(double* __restrict__ part, const cd* __restrict__ b, const cd* __restrict__ xv,
                                   const cd* __restrict__ U, const double* __restrict__ clov, Geom g, int bc_t,
                                   int nchunks) {
  __shared__ double sh[32 * 2];
  const int chunk = blockIdx.x, rhs = blockIdx.y;
  const int V = g.V;
  const cd* pb = b + (size_t)rhs * V * 12;
  const cd* px = xv + (size_t)rhs * V * 12;
  double rr = 0.0, bb = 0.0;
  for (int xi = chunk * blockDim.x + threadIdx.x; xi < V; xi += nchunks * blockDim.x) {
    int c[4];
    geom_coords(g, xi, c);
    cd acc[12], nb[12], u[9], d[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = czero<double>();
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
      int n[4] = {c[0], c[1], c[2], c[3]};
      n[mu] = (c[mu] + 1) % g.L[mu];
      double sgn = (mu == 0 && c[0] == g.L[0] - 1) ? double(bc_t) : 1.0;
      const cd* s1 = px + (size_t)lin4(n, g.L) * 12;
#pragma unroll
      for (int k = 0; k < 12; ++k) nb[k] = sgn * s1[k];
      load_link(U, V, mu, xi, u);
      hop_accumulate(mu, true, u, nb, acc);
      n[mu] = (c[mu] - 1 + g.L[mu]) % g.L[mu];
      sgn = (mu == 0 && c[0] == 0) ? double(bc_t) : 1.0;
      const cd* s2 = px + (size_t)lin4(n, g.L) * 12;
#pragma unroll
      for (int k = 0; k < 12; ++k) nb[k] = sgn * s2[k];
      load_link(U, V, mu, geom_index(g, n), u);
      hop_accumulate(mu, false, u, nb, acc);
    }
    const size_t lex = (size_t)lin4(c, g.L) * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) nb[k] = 1.0 * px[lex + k];
    clover_apply(clov, V, xi, nb, d);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const cd bk = pb[lex + k];
      const cd r = bk - (d[k] - 0.5 * acc[k]);
      rr += cnorm2(r);
      bb += cnorm2(bk);
    }
  }
  for (int off = 16; off >= 1; off >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, off);
    bb += __shfl_xor_sync(0xffffffffu, bb, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { sh[2 * warp] = rr; sh[2 * warp + 1] = bb; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, e = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += sh[2 * w]; e += sh[2 * w + 1]; }
    part[((size_t)rhs * nchunks + chunk) * 2] = a;
    part[((size_t)rhs * nchunks + chunk) * 2 + 1] = e;
  }
}

__global__ void k_resnorm_final(double* __restrict__ out, const double* __restrict__ part, int nchunks) {
  if (threadIdx.x != 0) return;
  const int rhs = blockIdx.x;
  double a = 0.0, e = 0.0;
  for (int c = 0; c < nchunks; ++c) {
    a += part[((size_t)rhs * nchunks + c) * 2];
    e += part[((size_t)rhs * nchunks + c) * 2 + 1];
  }
  out[rhs] = e > 0.0 ? sqrt(a) / sqrt(e) : 0.0;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
namespace dd {

void set_gamma_products(const double* gg /* [6][4][4][2] */) {
  cudaMemcpyToSymbol(c_gg, gg, sizeof(double) * 6 * 16 * 2);
}

template <typename T>
void fine_dslash(cplx<T>* out, const cplx<T>* in, const cplx<T>* b, const FineOp<T>& op, int nrhs,
                 size_t rstride, int sel, int sel_mu, int in_chir, cudaStream_t st) {
  dim3 grid(div_up(op.g.V, 128), nrhs);
  count_launch();
  if constexpr (sizeof(T) == 4) {
    if (op.Uh) {
      const float sh = op.shift;
      if (b)
        k_fine_dslash<float, true, __half2, __half2><<<grid, 128, 0, st>>>(out, in, b, op.Uh, op.clovh, op.g, op.bc_t,
                                                                          rstride, sel, sel_mu, in_chir, sh);
      else
        k_fine_dslash<float, false, __half2, __half2><<<grid, 128, 0, st>>>(out, in, b, op.Uh, op.clovh, op.g, op.bc_t,
                                                                           rstride, sel, sel_mu, in_chir, sh);
      return;
    }
  }
  if (b)
    k_fine_dslash<T, true, cplx<T>, T><<<grid, 128, 0, st>>>(out, in, b, op.U, op.clov, op.g, op.bc_t, rstride, sel,
                                                             sel_mu, in_chir, T(0));
  else
    k_fine_dslash<T, false, cplx<T>, T><<<grid, 128, 0, st>>>(out, in, b, op.U, op.clov, op.g, op.bc_t, rstride,
                                                              sel, sel_mu, in_chir, T(0));
}

// the staged kernel needs: FP32 compute, the SAP block tiling the aggregate
// (inner tile), 16-byte aligned component runs, and the staged block fitting in
// shared memory
template <typename T>
bool sap_tma_ok(const FineOp<T>& op) {
  if (sizeof(T) != 4) return false;
  for (int d = 0; d < 4; ++d)
    if (op.g.I[d] != op.g.B[d]) return false;
  const int q = op.Uh ? 8 : 4;
  if (op.g.vB % q || op.g.V % q || op.g.vB > 256) return false;
  return true;
}

template <typename T, typename LS, typename CS>
void launch_sap_tma(cplx<T>* z, const cplx<T>* b, const LS* U, const CS* clov, const FineOp<T>& op, const int* blocks,
                    int nblocks, int nrhs, size_t rstride, int k_mr, T shift, cudaStream_t st) {
  int seg = 1;
  while (seg < op.g.vB) seg <<= 1;
  const int threads = 256;
  const int segs = threads / seg;
  const size_t seg_bytes =
      (size_t)op.g.vB * (36 * sizeof(LS) + 2 * ClovRows<CS>::per_chir * sizeof(CS) + 12 * sizeof(cplx<T>));
  const size_t sm = segs * seg_bytes + 16 + (threads / 32) * 3 * sizeof(T) + 16;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_fine_sap_tma<T, LS, CS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr = true;
  }
  count_launch();
  k_fine_sap_tma<T, LS, CS><<<div_up(nblocks, segs), threads, sm, st>>>(z, b, U, clov, op.g, op.bc_t, rstride, nrhs,
                                                                       blocks, nblocks, seg, k_mr, op.err, shift);
}

// the 4^4 kernel: FP32 compute, 4^4 SAP blocks that are the inner tile (contiguous
// sites), and 16-byte aligned rows of z (bulk copies)
template <typename T>
bool sap_b4_ok(const FineOp<T>& op, const void* z, size_t rstride) {
  if (sizeof(T) != 4) return false;
  for (int d = 0; d < 4; ++d)
    if (op.g.B[d] != 4 || op.g.I[d] != 4) return false;
  return ((uintptr_t)z % 16) == 0 && rstride % 2 == 0 && op.g.V % 4 == 0;
}

template <typename LS, typename CS>
void launch_sap_b4(cplx<float>* z, const cplx<float>* b, const LS* U, const CS* clov, const FineOp<float>& op,
                   const int* blocks, int nblocks, int nrhs, size_t rstride, int k_mr, float shift, cudaStream_t st) {
  constexpr int VB = 256;
  const size_t sm = (size_t)VB * (36 * sizeof(LS) + 2 * ClovRows<CS>::per_chir * sizeof(CS) + 12 * sizeof(cplx<float>)) +
                    16 + 2 * 24 * sizeof(float);
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(k_fine_sap_b4<LS, CS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  });
  count_launch();
  // programmatic stream serialization: consecutive colour sweeps overlap the next sweep's operator
  // staging with the end of the previous one (the kernel waits for the previous grid before it
  // reads z or b)
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute pdl[1];
  pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  pdl[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.gridDim = dim3(nblocks, 1, 1);
  cfg.blockDim = dim3(VB, 1, 1);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cfg.attrs = pdl;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_fine_sap_b4<LS, CS>, z, b, U, clov, op.g, op.bc_t, rstride, nrhs, blocks, k_mr,
                         op.err, shift) != cudaSuccess) {
    cudaGetLastError();   // the attribute refused here: the same sweep as a plain launch
    k_fine_sap_b4<LS, CS><<<nblocks, VB, sm, st>>>(z, b, U, clov, op.g, op.bc_t, rstride, nrhs, blocks, k_mr, op.err,
                                                   shift);
  }
}

template <typename LS, typename CS>
void launch_sap_b4_eo(cplx<float>* z, const cplx<float>* b, const LS* U, const CS* mix, const FineOp<float>& op,
                      const int* blocks, int nblocks, int nrhs, size_t rstride, int k_mr, float shift,
                      cudaStream_t st) {
  constexpr int VB = 256;
  const size_t sm = (size_t)VB * (36 * sizeof(LS) + 2 * ClovRows<CS>::per_chir * sizeof(CS) + 12 * sizeof(cplx<float>)) +
                    (size_t)12 * 128 * sizeof(cplx<float>) + 16 + 2 * 12 * sizeof(float);
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(k_fine_sap_b4_eo<LS, CS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  });
  count_launch();
  k_fine_sap_b4_eo<LS, CS><<<nblocks, 128, sm, st>>>(z, b, U, mix, op.g, op.bc_t, rstride, nrhs, blocks, k_mr, op.err,
                                                     shift);
}

template <typename T, typename LS, typename CS>
void launch_sap_plain(cplx<T>* z, const cplx<T>* b, const LS* U, const CS* clov, const FineOp<T>& op,
                      const int* blocks, int nblocks, int nrhs, size_t rstride, int k_mr, T shift, cudaStream_t st) {
  int seg = 1;
  while (seg < op.g.vB) seg <<= 1;
  const int threads = seg >= 256 ? seg : 256;
  const int segs = threads / seg;
  const size_t sm = (size_t)threads * 12 * sizeof(cplx<T>) + (size_t)(threads / 32) * 3 * sizeof(T);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_fine_sap<T, LS, CS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  dim3 grid(div_up(nblocks, segs), nrhs);
  count_launch();
  k_fine_sap<T, LS, CS><<<grid, threads, sm, st>>>(z, b, U, clov, op.g, op.bc_t, rstride, blocks, nblocks, seg, k_mr,
                                                   shift);
}

template <typename T>
void fine_sap_sweep(cplx<T>* z, const cplx<T>* b, const FineOp<T>& op, const int* blocks, int nblocks, int nrhs,
                    size_t rstride, int k_mr, cudaStream_t st) {
  if (nrhs < 1 || nblocks < 1) return;   // the staged kernels issue their copies before the rhs loop
  const bool tma = sap_tma_ok(op) && op.err;
  if constexpr (sizeof(T) == 4) {
    if (op.schur && op.err && sap_b4_ok(op, z, rstride)) {
      // block solves on the even-odd Schur complement (per-site clover / inverse tables)
      if (op.Uh)
        launch_sap_b4_eo<__half2, __half2>(z, b, op.Uh, op.mixh, op, blocks, nblocks, nrhs, rstride, k_mr, op.shift,
                                           st);
      else
        launch_sap_b4_eo<cplx<float>, float>(z, b, op.U, op.mix32, op, blocks, nblocks, nrhs, rstride, k_mr, 0.f, st);
      return;
    }
    if (op.err && sap_b4_ok(op, z, rstride)) {
      if (op.Uh)
        launch_sap_b4<__half2, __half2>(z, b, op.Uh, op.clovh, op, blocks, nblocks, nrhs, rstride, k_mr, op.shift, st);
      else
        launch_sap_b4<cplx<float>, float>(z, b, op.U, op.clov, op, blocks, nblocks, nrhs, rstride, k_mr, 0.f, st);
      return;
    }
    if (op.Uh) {
      if (tma)
        launch_sap_tma<float, __half2, __half2>(z, b, op.Uh, op.clovh, op, blocks, nblocks, nrhs, rstride, k_mr,
                                               op.shift, st);
      else
        launch_sap_plain<float, __half2, __half2>(z, b, op.Uh, op.clovh, op, blocks, nblocks, nrhs, rstride, k_mr,
                                                 op.shift, st);
      return;
    }
  }
  if constexpr (sizeof(T) == 4) {   // the staged kernel is an FP32 kernel (sap_tma_ok)
    if (tma) {
      launch_sap_tma<T, cplx<T>, T>(z, b, op.U, op.clov, op, blocks, nblocks, nrhs, rstride, k_mr, T(0), st);
      return;
    }
  }
  launch_sap_plain<T, cplx<T>, T>(z, b, op.U, op.clov, op, blocks, nblocks, nrhs, rstride, k_mr, T(0), st);
}

__global__ void k_links_to_half(__half2* __restrict__ dst, const cplx<double>* __restrict__ U, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __halves2half2(__double2half(U[i].re), __double2half(U[i].im));
}

__global__ void k_clover_to_half(__half2* __restrict__ dst, const double* __restrict__ A, int V, double shift) {
  // row j of chirality ch holds the packed reals (2j, 2j+1); the diagonal (reals 0..5) loses the shift
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)36 * V) return;
  const int row = (int)(i / V), site = (int)(i - (size_t)row * V);
  const int ch = row / 18, p = 2 * (row - 18 * ch);
  const double a0 = A[(size_t)(ch * 36 + p) * V + site], a1 = A[(size_t)(ch * 36 + p + 1) * V + site];
  dst[i] = __halves2half2(__double2half(p < 6 ? a0 - shift : a0), __double2half(p + 1 < 6 ? a1 - shift : a1));
}

// out = Gamma_5 in (spins 2, 3 negated), component-major fine fields
__global__ void k_gamma5(cplx<double>* __restrict__ out, const cplx<double>* __restrict__ in, int V, size_t rstride) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)12 * V) return;
  const size_t a = (size_t)blockIdx.y * rstride + t;
  const cplx<double> v = in[a];
  out[a] = t < (size_t)6 * V ? v : cmk(-v.re, -v.im);
}

void fine_gamma5(cplx<double>* out, const cplx<double>* in, int V, int nrhs, size_t rstride, cudaStream_t st) {
  count_launch();
  k_gamma5<<<dim3(div_up((size_t)12 * V, 256), nrhs), 256, 0, st>>>(out, in, V, rstride);
}

void clover_inverse(double* inv, const double* clov, int V, int* err, cudaStream_t st) {
  count_launch();
  k_clover_inverse<<<div_up((size_t)2 * V, 128), 128, 0, st>>>(inv, clov, V, err);
}

void clover_mix(float* mix32, __half2* mixh, const double* clov, const double* inv, const Geom& g, double shift,
                cudaStream_t st) {
  if (mix32) {
    count_launch();
    k_clover_mix32<<<div_up((size_t)72 * g.V, 256), 256, 0, st>>>(mix32, clov, inv, g);
  }
  if (mixh) {
    count_launch();
    k_clover_mix_half<<<div_up((size_t)36 * g.V, 256), 256, 0, st>>>(mixh, clov, inv, g, shift);
  }
}

void double_to_df(dfl* dst, const double* src, size_t n, cudaStream_t st) {
  if (n == 0) return;
  count_launch();
  k_double_to_df<<<(unsigned)div_up(n, 256), 256, 0, st>>>(dst, src, n);
}

void fine_dslash_df(cplx<double>* out, const cplx<double>* in, const cplx<double>* b, const cplx<dfl>* Udf,
                    const dfl* clovdf, const Geom& g, int bc_t, int nrhs, size_t rstride, cudaStream_t st) {
  if (nrhs <= 0) return;
  const dim3 grid(div_up(g.V, 128), nrhs);
  count_launch();
  if (b) k_fine_dslash_df<true><<<grid, 128, 0, st>>>(out, in, b, Udf, clovdf, g, bc_t, rstride);
  else k_fine_dslash_df<false><<<grid, 128, 0, st>>>(out, in, b, Udf, clovdf, g, bc_t, rstride);
}

void links_to_half(__half2* dst, const cplx<double>* U, size_t n, cudaStream_t st) {
  count_launch();
  k_links_to_half<<<div_up(n, 256), 256, 0, st>>>(dst, U, n);
}

void clover_to_half(__half2* dst, const double* A, int V, double shift, cudaStream_t st) {
  count_launch();
  k_clover_to_half<<<div_up((size_t)36 * V, 256), 256, 0, st>>>(dst, A, V, shift);
}

void clover_build(double* clov, const cplx<double>* gauge_lex, const Geom& g, double m0, double csw,
                  cudaStream_t st) {
  count_launch();
  k_clover_build<<<div_up(g.V, 64), 64, 0, st>>>(clov, gauge_lex, g, m0, csw);
}

template <typename T>
void links_import(cplx<T>* U, const cplx<double>* gauge_lex, const Geom& g, cudaStream_t st) {
  count_launch();
  k_links_import<T><<<div_up(g.V, 128), 128, 0, st>>>(U, gauge_lex, g);
}

template <typename T>
void fine_import(cplx<T>* dst, const cplx<double>* src, const Geom& g, int nrhs, size_t rstride, cudaStream_t st) {
  count_launch();
  k_fine_import<T><<<dim3(div_up(g.V, 128), nrhs), 128, 0, st>>>(dst, src, g, rstride);
}

template <typename T>
void fine_export(cplx<double>* dst, const cplx<T>* src, const Geom& g, int nrhs, size_t rstride, cudaStream_t st) {
  count_launch();
  k_fine_export<T><<<dim3(div_up(g.V, 128), nrhs), 128, 0, st>>>(dst, src, g, rstride);
}

// device addresses of the allocation-free scratch, looked up once per device
static std::mutex g_noalloc_mu;
static double* g_noalloc_part_addr[64] = {};
static double* g_noalloc_out_addr[64] = {};

int fine_residual_norm_noalloc(double* out, bool out_on_device, const cplx<double>* b, const cplx<double>* x,
                               const FineOp<double>& op, int device, int nrhs, cudaStream_t st, const char** msg) {
  if (nrhs < 1 || nrhs > NOALLOC_MAX_RHS) {
    *msg = "n must be between 1 and 64 (the size of the static scratch)";
    return -1;
  }
  if (device < 0 || device >= 64) {
    *msg = "device index out of range";
    return -1;
  }
  // an error left on this thread by an earlier, unrelated call must not be reported as ours
  cudaGetLastError();
  // the scratch address is per device: look it up with the handle's device current, then
  // restore the caller's device
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    cudaGetLastError();
    *msg = "no usable current CUDA device";
    return -4;
  }
  const bool switch_dev = prev != device;
  if (switch_dev && cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    *msg = "cudaSetDevice to the handle's device failed";
    return -4;
  }
  int rc = 0;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_part_addr[device]) {
      double* p = nullptr;
      double* o = nullptr;
      if (cudaGetSymbolAddress((void**)&p, g_noalloc_partials) != cudaSuccess ||
          cudaGetSymbolAddress((void**)&o, g_noalloc_out) != cudaSuccess) {
        cudaGetLastError();
        *msg = "cudaGetSymbolAddress of the static scratch failed";
        rc = -4;
      } else {
        g_noalloc_part_addr[device] = p;
        g_noalloc_out_addr[device] = o;
      }
    }
  }
  if (rc == 0) {
    int nchunks = (op.g.V + 255) / 256;
    if (nchunks > NOALLOC_CHUNKS) nchunks = NOALLOC_CHUNKS;
    double* dst = out_on_device ? out : g_noalloc_out_addr[device];
    count_launch(2);
    k_resnorm_partials<<<dim3(nchunks, nrhs), 256, 0, st>>>(g_noalloc_part_addr[device], b, x, op.U, op.clov, op.g,
                                                            op.bc_t, nchunks);
    if (cudaPeekAtLastError() != cudaSuccess) {
      *msg = "launch of the residual kernel failed";
      rc = -4;
    }
    if (rc == 0) {
      k_resnorm_final<<<nrhs, 32, 0, st>>>(dst, g_noalloc_part_addr[device], nchunks);
      if (cudaPeekAtLastError() != cudaSuccess) {
        *msg = "launch of the reduction kernel failed";
        rc = -4;
      }
    }
    if (rc == 0 && !out_on_device &&
        cudaMemcpyAsync(out, dst, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
      *msg = "copy of the result to the host failed";
      rc = -4;
    }
    if (rc == 0 && cudaStreamSynchronize(st) != cudaSuccess) {
      *msg = "kernel failure";
      rc = -4;
    }
    if (rc != 0) cudaGetLastError();
  }
  if (switch_dev) cudaSetDevice(prev);
  return rc;
}

#define INST(T)                                                                                              \
  template void fine_dslash<T>(cplx<T>*, const cplx<T>*, const cplx<T>*, const FineOp<T>&, int, size_t, int, \
                               int, int, cudaStream_t);                                                      \
  template void fine_sap_sweep<T>(cplx<T>*, const cplx<T>*, const FineOp<T>&, const int*, int, int, size_t, \
                                  int, cudaStream_t);                                                        \
  template void links_import<T>(cplx<T>*, const cplx<double>*, const Geom&, cudaStream_t);                  \
  template void fine_import<T>(cplx<T>*, const cplx<double>*, const Geom&, int, size_t, cudaStream_t);      \
  template void fine_export<T>(cplx<double>*, const cplx<T>*, const Geom&, int, size_t, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace dd
