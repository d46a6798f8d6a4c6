// Coarse stencil on tensor cores: (D phi)(A) = S(A) phi(A) + sum_mu [F_mu(A) phi(A+mu) + B_mu(A) phi(A-mu)]
// (the Galerkin operator of Sec. 1, a 9-point stencil of dense n x n complex blocks) for a batch of
// right-hand sides, written per coarse site A as one small GEMM
//   Y (n x R) = [S | F_t .. F_x | B_t .. B_x] (n x 9n)  *  [phi(A); phi(A+t); ..; phi(A-x)] (9n x R)
// so the site's blocks are read from memory once for the whole batch.
//
// Precision (FP32 arithmetic on FP16 storage): the blocks are the stored FP16 values (one FP32 scale
// per site, applied to the result); each right-hand side's staged neighbour values are scaled by a
// power of two s_r >= max |Re|, |Im| (exact) and split into FP16 hi + lo parts (x/s_r = hi + lo to
// about 2^-23 s_r), multiplied on the tensor cores (mma.sync m16n8k16, FP16 in, FP32 accumulate) in
// the real form of the complex product:
//   [Re y; Im y] rows 2i, 2i+1  =  [[Re a, -Im a], [Im a, Re a]]  *  [Re x; Im x] rows 2j, 2j+1.
// A column's result depends only on that column's values and scale (no cross-column reduction), so a
// right-hand side gives the same bits alone and inside any batch.
//
// Layout: one CTA per (coarse site, group of up to 16 right-hand sides); the site's 9 blocks
// (column-major, contiguous: element (i, j) of block k at (k n + j) n + i) are staged whole by one
// bulk copy; warp w computes the 16-row tile w % MT of the 2n real rows over the k-tiles of its
// share w / MT of the 9n complex columns (ks shares, reduced in a fixed order).
#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

#include <atomic>
#include <mutex>

namespace {

constexpr int TC_R = 16;   // right-hand sides per CTA (two 8-column MMA tiles)

__device__ __forceinline__ void mma_16816(float c[4], const unsigned a[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct TcLayout {
  int mt;       // 16-row tiles of the 2n real rows
  int kcp;      // complex columns padded to whole k-tiles (8 complex = 16 real)
  int xs;       // row stride (8-byte slots) of the staged vectors: = 4 mod 16 spreads the banks
  size_t off_x, off_y, off_red, total;
};

__host__ __device__ inline TcLayout tc_layout(int n, int ks) {
  TcLayout L;
  L.mt = (2 * n + 15) / 16;
  L.kcp = ((9 * n + 7) / 8) * 8;
  L.xs = L.kcp + ((L.kcp % 16) == 0 ? 4 : 12);
  L.off_x = (size_t)36 * n * n;                                  // 9 n^2 half2 (a multiple of 16 bytes)
  L.off_y = L.off_x + (size_t)TC_R * L.xs * 8;                    // {hi, lo} half2 pairs
  L.off_red = L.off_y + (size_t)TC_R * n * 8;                     // complex float results
  L.total = L.off_red + (size_t)(ks > 1 ? ks - 1 : 0) * L.mt * 32 * 8 * sizeof(float);
  return L;
}

template <bool RESID>
__global__ void k_coarse_apply_tc(cplx<float>* __restrict__ out, const cplx<float>* __restrict__ in,
                                  const cplx<float>* __restrict__ bsrc, const __half2* __restrict__ blk,
                                  const float* __restrict__ bscale, Geom g, int n, size_t rstride, int nrhs, int ks,
                                  int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ int nbr[9];
  __shared__ unsigned smax[TC_R];
  __shared__ float sscale[TC_R];
  const TcLayout Lo = tc_layout(n, ks);
  const __half2* sA = reinterpret_cast<const __half2*>(smem);
  uint2* sX = reinterpret_cast<uint2*>(smem + Lo.off_x);       // float2 staging, then {hi, lo}
  float* sY = reinterpret_cast<float*>(smem + Lo.off_y);       // [r][i][re, im]
  float* sRed = reinterpret_cast<float*>(smem + Lo.off_red);
  const int site = blockIdx.x;
  const int r0 = blockIdx.y * TC_R;
  const int nr = min(TC_R, nrhs - r0);
  const int tid = threadIdx.x, nth = blockDim.x;
  const unsigned abytes = (unsigned)(36 * n * n);
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_arrive_expect_tx(&bar, abytes);
    bulk_g2s(smem, blk + (size_t)site * 9 * n * n, abytes, &bar);
  }
  if (tid < 9) {
    int c[4];
    geom_coords(g, site, c);
    nbr[tid] = tid == 0 ? site : geom_neighbor(g, c, (tid - 1) % 4, tid <= 4 ? +1 : -1);
  }
  if (tid < TC_R) smax[tid] = 0u;
  __syncthreads();
  // stage the neighbour values of every column (zero beyond the batch and the padding); the column's
  // max |Re|, |Im| is reduced per warp by shuffles, then one shared-memory atomic per warp and column
  const int kc = 9 * n;
  for (int r = 0; r < TC_R; ++r) {
    float m = 0.f;
    float2* dst = reinterpret_cast<float2*>(sX) + (size_t)r * Lo.xs;
    for (int cc = tid; cc < Lo.kcp; cc += nth) {
      float2 v = make_float2(0.f, 0.f);
      if (r < nr && cc < kc) {
        const int k = cc / n;
        const cplx<float> x = in[(size_t)(r0 + r) * rstride + (size_t)nbr[k] * n + (cc - k * n)];
        v = make_float2(x.re, x.im);
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
      dst[cc] = v;
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((tid & 31) == 0 && m > 0.f) atomicMax(&smax[r], __float_as_uint(m));   // order-independent
  }
  __syncthreads();
  if (tid < TC_R) {
    const float m = __uint_as_float(smax[tid]);
    int ex = 0;
    frexpf(m, &ex);                                  // m = f 2^ex, f in [0.5, 1): 2^ex >= m
    sscale[tid] = m > 0.f ? ldexpf(1.f, ex) : 1.f;
  }
  __syncthreads();
  // split in place: x / s = hi + lo, both FP16 (the slot of an entry is owned by one thread)
  for (int r = 0; r < TC_R; ++r) {
    const float inv = 1.f / sscale[r];               // exact: a power of two
    uint2* row = sX + (size_t)r * Lo.xs;
    for (int cc = tid; cc < Lo.kcp; cc += nth) {
      const float2 v = reinterpret_cast<float2*>(row)[cc];
      const float xr = v.x * inv, xi = v.y * inv;
      const __half2 hi = __floats2half2_rn(xr, xi);
      const float2 hf = __half22float2(hi);
      const __half2 lo = __floats2half2_rn(xr - hf.x, xi - hf.y);
      uint2 u;
      u.x = *reinterpret_cast<const unsigned*>(&hi);
      u.y = *reinterpret_cast<const unsigned*>(&lo);
      row[cc] = u;
    }
  }
  const bool ok = __syncthreads_and(mbar_wait_bounded(&bar, 0) ? 1 : 0);
  if (!ok) {
    // staging wait ran out: flag it, let the copy in flight land (bounded) and leave
    if (tid == 0) {
      if (err) atomicExch(err, 2);
      mbar_wait_bounded(&bar, 0);
    }
    return;
  }
  const int warp = tid >> 5, lane = tid & 31;
  const int mtile = warp % Lo.mt, kq = warp / Lo.mt;
  const int gq = lane >> 2, tq = lane & 3;
  const int KT = Lo.kcp / 8;
  const int kt0 = (kq * KT) / ks, kt1 = ((kq + 1) * KT) / ks;
  const int nt = nr > 8 ? 2 : 1;
  const int ia = mtile * 8 + (gq >> 1), ib = ia + 4;
  const bool imrow = (gq & 1) != 0;
  const unsigned* sAu = reinterpret_cast<const unsigned*>(sA);
  // FP32 accumulators: the hi products in four chains (k-tile mod 4), the lo products in their own;
  // the tensor core's accumulation truncates, so short chains keep its bias from adding up along K
  float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  float ach[4][2][4] = {};
  // A-fragment word of complex element (i, cc): (Re a, -Im a) on a real-part row, (Im a, Re a) on an
  // imaginary-part row; zero outside the n x 9n matrix
  auto afrag = [&](int i, int cc) -> unsigned {
    if (i >= n || cc >= kc) return 0u;
    const unsigned w = sAu[(size_t)cc * n + i];
    return imrow ? __byte_perm(w, 0, 0x1032) : (w ^ 0x80000000u);
  };
  for (int kt = kt0; kt < kt1; ++kt) {
    const int c0 = kt * 8 + tq, c1 = c0 + 4;
    unsigned a[4];
    a[0] = afrag(ia, c0);
    a[1] = afrag(ib, c0);
    a[2] = afrag(ia, c1);
    a[3] = afrag(ib, c1);
    const int ch = kt & 3;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q < nt) {
        const int r = q * 8 + gq;
        const uint2 x0 = sX[r * Lo.xs + c0];
        const uint2 x1 = sX[r * Lo.xs + c1];
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (c == ch) mma_16816(ach[c][q], a, x0.x, x1.x);
        mma_16816(acc[q], a, x0.y, x1.y);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[q][v] = ((ach[0][q][v] + ach[1][q][v]) + (ach[2][q][v] + ach[3][q][v])) + acc[q][v];
  // fixed-order reduction of the k shares
  if (ks > 1) {
    if (kq > 0) {
      float* dst = sRed + ((size_t)((kq - 1) * Lo.mt + mtile) * 32 + lane) * 8;
#pragma unroll
      for (int q = 0; q < 8; ++q) dst[q] = acc[q >> 2][q & 3];
    }
    __syncthreads();
    if (kq == 0)
      for (int s = 1; s < ks; ++s) {
        const float* src = sRed + ((size_t)((s - 1) * Lo.mt + mtile) * 32 + lane) * 8;
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q >> 2][q & 3] += src[q];
      }
  }
  if (kq == 0) {
    const float bs = bscale ? bscale[site] : 1.f;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q >= nt) continue;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int row = mtile * 16 + gq + (v >= 2 ? 8 : 0);
        const int col = q * 8 + 2 * tq + (v & 1);
        const int i = row >> 1;
        if (i < n && col < nr) sY[((size_t)col * n + i) * 2 + (row & 1)] = (acc[q][v] * sscale[col]) * bs;
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < nr * n; e += nth) {
    const int r = e / n, i = e - r * n;
    const size_t a = (size_t)(r0 + r) * rstride + (size_t)site * n + i;
    const cplx<float> y = cmk<float>(sY[2 * e], sY[2 * e + 1]);
    out[a] = RESID ? bsrc[a] - y : y;
  }
}

// The dynamic shared-memory limit is a process-wide attribute of the kernel: it only ever grows
// (under a lock, so that two threads preparing different sizes cannot leave it at the smaller)
template <bool RESID>
cudaError_t prepare_tc(size_t bytes) {
  static std::atomic<size_t> set_to{0};
  static std::mutex mu;
  if (set_to.load(std::memory_order_acquire) >= bytes) return cudaSuccess;
  std::lock_guard<std::mutex> lk(mu);
  if (set_to.load(std::memory_order_relaxed) >= bytes) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(k_coarse_apply_tc<RESID>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) set_to.store(bytes, std::memory_order_release);
  return e;
}

}  // namespace

namespace dd {

size_t coarse_tc_smem(int n, int ks) { return tc_layout(n, ks).total; }

// largest CTA both variants can launch with their register counts (queried once)
int tc_max_threads() {
  static std::atomic<int> cached{0};
  int v = cached.load(std::memory_order_acquire);
  if (v > 0) return v;
  cudaFuncAttributes a0, a1;
  if (cudaFuncGetAttributes(&a0, k_coarse_apply_tc<false>) != cudaSuccess ||
      cudaFuncGetAttributes(&a1, k_coarse_apply_tc<true>) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  v = a0.maxThreadsPerBlock < a1.maxThreadsPerBlock ? a0.maxThreadsPerBlock : a1.maxThreadsPerBlock;
  cached.store(v, std::memory_order_release);
  return v;
}

bool coarse_tc_fits(int n, int ks) {
  // bulk copy of one site's blocks: at most 2^20 - 1 bytes on one mbarrier; 227 KB of shared memory;
  // the CTA (one warp per 16-row tile and k-split) within what the kernel's registers allow
  const TcLayout L = tc_layout(n, ks);
  return ks >= 1 && ks <= 4 && (size_t)36 * n * n < (1u << 20) && L.total + 512 <= 227 * 1024 &&
         32 * L.mt * ks <= tc_max_threads();
}

cudaError_t coarse_apply_tc(cplx<float>* out, const cplx<float>* in, const cplx<float>* b, const CoarseOp<float>& op,
                            int nrhs, size_t rstride, int ks, cudaStream_t st) {
  if (nrhs <= 0) return cudaSuccess;
  if (!op.blkh || !coarse_tc_fits(op.n, ks)) return cudaErrorInvalidValue;
  const TcLayout L = tc_layout(op.n, ks);
  const dim3 grid(op.g.V, (nrhs + TC_R - 1) / TC_R);
  const int threads = 32 * L.mt * ks;
  count_launch();
  if (b) {
    const cudaError_t e = prepare_tc<true>(L.total);
    if (e != cudaSuccess) return e;
    k_coarse_apply_tc<true><<<grid, threads, L.total, st>>>(out, in, b, op.blkh, op.bscale, op.g, op.n, rstride,
                                                            nrhs, ks, op.err);
  } else {
    const cudaError_t e = prepare_tc<false>(L.total);
    if (e != cudaSuccess) return e;
    k_coarse_apply_tc<false><<<grid, threads, L.total, st>>>(out, in, b, op.blkh, op.bscale, op.g, op.n, rstride,
                                                             nrhs, ks, op.err);
  }
  return cudaPeekAtLastError();
}

}  // namespace dd
