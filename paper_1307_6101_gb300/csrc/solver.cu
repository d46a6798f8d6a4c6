// Host orchestration of the DD-alpha-AMG method and the C ABI (include/ddamg.h).
//
// Paper references: the cycle is Alg. 2 (the K-cycle: Alg. 1 with the
// recursion replaced by FGMRES on D_{l+1} preconditioned by the K-cycle at
// l+1), the setup is Alg. 3 followed by n_inv applications of Alg. 4, the
// outer solver is FP64 FGMRES (Sec. 3), the coarsest system is solved by
// odd-even preconditioned GMRES to relative accuracy epsilon (Sec. 3), and the
// parameters default to Table 1.  Every arithmetic step runs in the CUDA
// kernels of this library; the host only sequences launches and reads one
// small per-rhs status array per Krylov iteration.
#include "ddamg.h"
#include "kernels.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

using namespace dd;

namespace {

thread_local std::string g_err;

struct DdError {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, const std::string& m) { throw DdError{code, m}; }

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) fail(DDAMG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
struct Work {
  cplx<T>* bc = nullptr;   // right-hand side of this level's inner solve
  cplx<T>* xs = nullptr;   // result of this level's inner solve (last iterate of the level)
  cplx<T>* V = nullptr;    // Krylov basis [m+1][max_rhs][vlen]
  cplx<T>* Z = nullptr;    // preconditioned vectors [m][max_rhs][vlen] (flexible only)
  cplx<T>* r = nullptr;    // residual
  cplx<T>* t[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  cplx<T>* cur = nullptr;  // current basis vector (device-driven solver)
  cplx<T>* zc = nullptr;   // preconditioned current vector (device-driven solver)
  cplx<T>* wv = nullptr;   // new Krylov direction (device-driven solver)
  cplx<T>* gin = nullptr;  // fixed input of a captured K-cycle starting on this level
  cplx<T>* gout = nullptr; // fixed output of a captured K-cycle starting on this level
  GmresState gs{};
  int m = 0;
  int batch = 0;              // columns the vectors hold (stride of the Krylov basis: batch * vlen)
  long long host_steps = 0;   // Arnoldi steps taken by the host-driven solver
};

struct Level {
  int idx = 0;
  bool fine = false, coarsest = false;
  Geom g{};
  int n = 0;          // dof per site
  size_t vlen = 0;    // complex elements per field
  int N = 0;          // test vectors (columns of P per chirality)
  FineOp<double> f64{};
  FineOp<float> f32{};
  CoarseOp<double> c64{};
  CoarseOp<float> c32{};
  cplx<double>* tv64 = nullptr;
  cplx<double>* P64 = nullptr;
  cplx<float>* P32 = nullptr;
  // FP16 storage copies read by the FP32 kernels when the handle stores FP16
  __half2* Uh = nullptr;      // fine links
  __half2* clovh = nullptr;   // fine clover term without the (m0 + 4) shift (pairs of packed reals)
  __half2* Ph = nullptr;      // P_l, one scale per (aggregate, chirality) in pscale
  float* pscale = nullptr;
  __half2* blkh = nullptr;    // coarse blocks, one scale per site in bscale
  float* bscale = nullptr;
  float* mix32 = nullptr;     // fine level, Schur SAP: clover (even sites) / inverse (odd sites), FP32
  cplx<dfl>* Udf = nullptr;   // fine level: links as double-FP32 pairs (outer operator option)
  dfl* clovdf = nullptr;      // fine level: (m0 + 4) + clover as double-FP32 pairs
  __half2* mixh = nullptr;    // the same tables in FP16
  int* blocks[2] = {nullptr, nullptr};
  int nblocks[2] = {0, 0};
  int* bsite = nullptr;       // coarse levels: [nBlk][vB] site of each SAP block's sites (block-local order)
  int* bloc = nullptr;        // coarse levels: [V] position of each site inside its SAP block
  bool eo = true;             // coarsest level: odd-even solve possible (even extents)
  int tr_ks = 0;              // restriction to l+1 on FP16 P: 0 per-rhs kernel, k tensor cores with k-split k
  int pr_batch = 0;           // prolongation from l+1 on FP16 P: 1 = the batch kernel (P read once)
  int sap_persist = 0;        // coarse levels on FP16 blocks: 1 = a smoother call is one persistent launch
  int sap_nbpc = 0;           // SAP blocks of each colour per cluster of that launch (1 or 2)
  unsigned* sap_gcnt = nullptr;   // barrier counter of that launch
  Work<double> w64;
  Work<float> w32;
};

template <typename T> FineOp<T>& fop(Level& L);
template <> FineOp<double>& fop<double>(Level& L) { return L.f64; }
template <> FineOp<float>& fop<float>(Level& L) { return L.f32; }
template <typename T> CoarseOp<T>& cop(Level& L);
template <> CoarseOp<double>& cop<double>(Level& L) { return L.c64; }
template <> CoarseOp<float>& cop<float>(Level& L) { return L.c32; }
template <typename T> Work<T>& work(Level& L);
template <> Work<double>& work<double>(Level& L) { return L.w64; }
template <> Work<float>& work<float>(Level& L) { return L.w32; }
template <typename T> cplx<T>* Pptr(Level& L);
template <> cplx<double>* Pptr<double>(Level& L) { return L.P64; }
template <> cplx<float>* Pptr<float>(Level& L) { return L.P32; }

struct Scratch {
  void* p = nullptr;
  size_t cap = 0;
};

// stream capture of a K-cycle into a CUDA graph; bodies of conditional nodes are
// captured on deeper streams
struct CaptureCtx {
  bool active = false;
  int depth = 0;
  cudaStream_t s[12] = {};
};

struct GraphEntry {
  int l0 = 0, tsize = 0, nrhs = 0, prof = 0;
  cudaGraphExec_t exec = nullptr;
  std::vector<int> ev_kind;
  std::vector<double> ev_bytes;
  std::vector<cudaEvent_t> ev;   // pairs
};

}  // namespace

struct ddamg_handle {
  ddamg_params p{};
  int device = 0;
  size_t dev_bytes = 0;   // bytes of the library's own device allocations for this handle
  // wall-clock seconds of the setup per level and phase (DDAMG_SETUP_* order)
  double setup_s[DDAMG_MAX_LEVELS][DDAMG_SETUP_KINDS] = {};
  int dims[4] = {0, 0, 0, 0};
  int bc_t = -1;
  double m0 = 0, csw = 0;
  int L = 0;
  std::vector<Level> lv;
  cudaStream_t own = nullptr;
  cudaStream_t st = nullptr;
  std::vector<void*> allocs;
  Scratch scr[8];
  // outer FGMRES (FP64, level 0)
  Work<double> outer;
  cplx<double>* ob = nullptr;
  cplx<double>* ox = nullptr;
  cplx<float>* pin32 = nullptr;
  cplx<float>* pout32 = nullptr;
  int* d_err = nullptr;
  int* h_done = nullptr;      // pinned
  double* h_scal = nullptr;   // pinned
  int* h_kr = nullptr;        // pinned
  int max_batch = 0;          // right-hand sides per solve batch (params.max_rhs)
  int work_batch = 0;         // columns of the level workspaces: max(max_rhs, setup batch of Alg. 4)
  // per-kernel-class CUDA-event timing (ddamg_profile)
  int prof = 0;   // bitmask of recorded kernel classes
  std::vector<cudaEvent_t> ev[DDAMG_PROF_KINDS];
  size_t ev_used[DDAMG_PROF_KINDS] = {};
  double prof_bytes[DDAMG_PROF_KINDS] = {};
  long long prof_count[DDAMG_PROF_KINDS] = {};
  double prof_graph_ms[DDAMG_PROF_KINDS] = {};
  // CUDA graphs of K-cycles (device-driven inner solves)
  bool use_graphs = true;
  CaptureCtx cap;
  std::vector<GraphEntry*> graphs;
  GraphEntry* capturing = nullptr;
  cplx<double>* pin64 = nullptr;
  cplx<double>* pout64 = nullptr;
  // FP16 storage of links, clover term, P and coarse blocks under FP32 arithmetic
  bool half = false;
  bool work_ready[2] = {false, false};   // Work<double>, Work<float> allocated on every level
  // autotuner of the coarse stencil kernels: milliseconds per application at the batch size for
  // [level][candidate] (candidate 0 = CUDA-core kernel, k = tensor cores with k-split k; -1 = not run)
  double tune_ms[4][DDAMG_MAX_LEVELS][5] = {};   // [DDAMG_TUNE_*][level][candidate]
  int tc_force = -1;   // DDAMG_OPT_COARSE_TC: -1 autotune, 0 CUDA cores, k >= 1 that split
  int persist_force = -1;   // DDAMG_OPT_SAP_PERSIST: -1 autotune, 0 per-sweep launches, 1 persistent,
                            // 2 persistent with two SAP blocks of each colour per cluster
  bool outer_df = false;    // DDAMG_OPT_OUTER_DF: outer D z_j and Gram-Schmidt in double-FP32 arithmetic
  bool sap_schur = false;   // fine-level FP32 SAP block solves on the even-odd Schur complement
  int setup_batch = 4;      // test vectors per batched K-cycle of Alg. 4
  // plain Krylov solver (CGNR) and sigma_min: four FP64 fine vectors per batch column, per-column
  // coefficients on the device, pinned host scalars
  cplx<double>* cg_vec = nullptr;
  cplx<double>* cg_coef = nullptr;
  double* cg_dcoef = nullptr;
  double* cg_host = nullptr;
  // coarsest level on a thread-block cluster
  bool use_cluster = true;
  CoarsestGeo cgeo;
  CoarsestPlan cplan32, cplan64;
  bool have_cplan32 = false, have_cplan64 = false;
};

namespace {

template <typename T>
T* dalloc(ddamg_handle* h, size_t count) {
  void* p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(&p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(DDAMG_ERR_OOM, "device allocation of " + std::to_string(count * sizeof(T)) + " bytes failed");
  }
  h->allocs.push_back(p);
  h->dev_bytes += count * sizeof(T);
  return static_cast<T*>(p);
}

void* scratch(ddamg_handle* h, int slot, size_t bytes) {
  Scratch& s = h->scr[slot];
  if (bytes > s.cap) {
    if (s.p) {
      CK(cudaStreamSynchronize(h->st));
      cudaFree(s.p);
      s.p = nullptr;
      h->dev_bytes -= s.cap;
      s.cap = 0;
    }
    if (cudaMalloc(&s.p, bytes) != cudaSuccess) {
      cudaGetLastError();
      fail(DDAMG_ERR_OOM, "scratch allocation of " + std::to_string(bytes) + " bytes failed");
    }
    h->dev_bytes += bytes;
    s.cap = bytes;
  }
  return s.p;
}

void sync(ddamg_handle* h) {
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->st));
}

// record an event pair around one launch of kind k when profiling; bytes = its algorithmic bytes
struct Prof {
  ddamg_handle* h;
  int k;
  size_t i;
  bool on;
  Prof(ddamg_handle* hh, int kind, double bytes) : h(hh), k(kind), i(0), on(((hh->prof >> kind) & 1) != 0) {
    if (!on) return;
    if (h->cap.active) {
      // inside a captured graph: event nodes only at the top level (not inside conditional bodies)
      if (h->cap.depth > 0 || !h->capturing) {
        on = false;
        return;
      }
      GraphEntry* e = h->capturing;
      cudaEvent_t a, b;
      CK(cudaEventCreate(&a));
      CK(cudaEventCreate(&b));
      i = e->ev.size();
      e->ev.push_back(a);
      e->ev.push_back(b);
      e->ev_kind.push_back(k);
      e->ev_bytes.push_back(bytes);
      CK(cudaEventRecordWithFlags(a, h->st, cudaEventRecordExternal));   // an event node, not a capture join
      return;
    }
    auto& v = h->ev[k];
    i = h->ev_used[k];
    while (v.size() < i + 2) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      v.push_back(e);
    }
    h->ev_used[k] = i + 2;
    h->prof_bytes[k] += bytes;
    h->prof_count[k] += 1;
    CK(cudaEventRecord(v[i], h->st));
  }
  ~Prof() {
    if (!on) return;
    if (h->cap.active) cudaEventRecordWithFlags(h->capturing->ev[i + 1], h->st, cudaEventRecordExternal);
    else cudaEventRecord(h->ev[k][i + 1], h->st);
  }
};

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// device view of a caller buffer of `bytes` (copied to staging slot if host)
const void* dev_in(ddamg_handle* h, const void* p, size_t bytes, int slot) {
  if (is_device_ptr(p)) return p;
  void* d = scratch(h, slot, bytes);
  CK(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, h->st));
  return d;
}

// ---------------------------------------------------------------------------
// operators on one level
template <typename T>
void apply_D(ddamg_handle* h, Level& L, cplx<T>* out, const cplx<T>* in, const cplx<T>* b, int nrhs,
             int sel = SEL_FULL, int mu = 0, int chir = -1) {
  const double cs = 2.0 * sizeof(T);
  const double vec = (double)L.vlen * cs * nrhs * (b ? 3 : 2);
  // operator data in its storage format: FP16 copies (4 bytes per complex, 2 per real) when in use
  const bool hf = sizeof(T) == 4 && h->half;
  const double os = hf ? 4.0 : cs, rs = hf ? 2.0 : (double)sizeof(T);
  if (L.fine) {
    Prof pr(h, DDAMG_PROF_FINE_DSLASH, vec + (double)L.g.V * (36 * os + 72 * rs));
    fine_dslash<T>(out, in, b, fop<T>(L), nrhs, L.vlen, sel, mu, chir, h->st);
  } else {
    Prof pr(h, DDAMG_PROF_COARSE_APPLY, vec + (double)L.g.V * 9 * L.n * L.n * os);
    coarse_apply<T>(out, in, b, cop<T>(L), nrhs, L.vlen, sel, mu, chir, h->st);
  }
}

// algorithmic bytes of one SAP colour sweep: per site of the colour b, z in, z out
// and the operator once; per block the neighbour values across its faces (and
// on the fine level the links of the backward hops entering the block)
template <typename T>
double sap_bytes(const Level& L, int c, int nrhs, bool half) {
  const double cs = 2.0 * sizeof(T);
  const double os = half ? 4.0 : cs;                   // bytes of one stored operator complex
  const double rs = half ? 2.0 : (double)sizeof(T);    // bytes of one stored operator real
  const double nsite = (double)L.nblocks[c] * L.g.vB;
  double faces = 0;
  for (int d = 0; d < 4; ++d) faces += (double)L.g.vB / L.g.B[d];
  if (L.fine)
    return nsite * (nrhs * 36 * cs + 36 * os + 72 * rs) + L.nblocks[c] * (nrhs * 2 * faces * 12 * cs + faces * 9 * os);
  return nsite * (nrhs * 3.0 * L.n * cs + 9.0 * L.n * L.n * os + (half ? 4.0 : 0.0)) +
         L.nblocks[c] * nrhs * 2 * faces * L.n * cs;
}

template <typename T> bool half_on(const ddamg_handle* h) { return sizeof(T) == 4 && h->half; }

// iterations x { z <- z + M_SAP (b - D z) }: each SAP application is a red then a black sweep
template <typename T>
void sap(ddamg_handle* h, Level& L, cplx<T>* z, const cplx<T>* b, int nrhs, int iterations) {
  if constexpr (sizeof(T) == 4) {
    if (!L.fine && L.sap_persist && L.c32.sap_cls > 0 && half_on<T>(h) && iterations > 0) {
      // every sweep of the call in one launch (the tuner checked that it runs, eagerly and in a graph)
      Prof pr(h, DDAMG_PROF_COARSE_SAP,
              iterations * (sap_bytes<T>(L, 0, nrhs, true) + sap_bytes<T>(L, 1, nrhs, true)));
      CK(coarse_sap_persist(z, b, L.c32, L.blocks[0], L.nblocks[0], L.blocks[1], L.nblocks[1], nrhs, L.vlen,
                            h->p.mr_steps, iterations, L.sap_nbpc, L.sap_gcnt, h->st));
      return;
    }
  }
  for (int it = 0; it < iterations; ++it)
    for (int c = 0; c < 2; ++c) {
      if (L.nblocks[c] == 0) continue;
      Prof pr(h, L.fine ? DDAMG_PROF_FINE_SAP : DDAMG_PROF_COARSE_SAP, sap_bytes<T>(L, c, nrhs, half_on<T>(h)));
      if (L.fine)
        fine_sap_sweep<T>(z, b, fop<T>(L), L.blocks[c], L.nblocks[c], nrhs, L.vlen, h->p.mr_steps, h->st);
      else
        CK(coarse_sap_sweep<T>(z, b, cop<T>(L), L.blocks[c], L.nblocks[c], nrhs, L.vlen, h->p.mr_steps, h->st));
    }
}

template <typename T>
void restrict_lv(ddamg_handle* h, int l, cplx<T>* out, const cplx<T>* in, int nrhs) {
  Level& F = h->lv[l];
  Level& C = h->lv[l + 1];
  const double cs = 2.0 * sizeof(T);
  const bool hf = half_on<T>(h);
  const double ps = hf ? 4.0 : cs;
  Prof pr(h, DDAMG_PROF_TRANSFER, (double)F.vlen * (cs * nrhs + ps * F.N) + (double)C.vlen * cs * nrhs);
  restrict_op<T>(out, in, Pptr<T>(F), F.g, C.g, F.fine, F.n, F.N, nrhs, F.vlen, C.vlen, C.n, h->st,
                 hf ? F.Ph : nullptr, hf ? F.pscale : nullptr, hf ? F.tr_ks : 0);
}

template <typename T>
void prolong_lv(ddamg_handle* h, int l, cplx<T>* out, const cplx<T>* in, int nrhs, bool acc) {
  Level& F = h->lv[l];
  Level& C = h->lv[l + 1];
  const double cs = 2.0 * sizeof(T);
  const bool hf = half_on<T>(h);
  const double ps = hf ? 4.0 : cs;
  Prof pr(h, DDAMG_PROF_TRANSFER,
          (double)F.vlen * (cs * nrhs * (acc ? 2 : 1) + ps * F.N) + (double)C.vlen * cs * nrhs);
  prolong_op<T>(out, in, Pptr<T>(F), F.g, C.g, F.fine, F.n, F.N, nrhs, F.vlen, C.vlen, acc, h->st,
                hf ? F.Ph : nullptr, hf ? F.pscale : nullptr, hf ? F.pr_batch : 0);
}

// ---------------------------------------------------------------------------
// (F)GMRES with per-rhs stopping (Saad's FGMRES with CGS2 Arnoldi and Givens
// rotations).  A(out, in, b): out = A in, or out = b - A in when b != null.
// M(out, in): preconditioner (flexible only).
struct KrylovResult {
  std::vector<int> iterations, cycles, converged;
  std::vector<double> true_residual;
};

template <typename T, class AOp, class MOp>
void krylov_host(ddamg_handle* h, Work<T>& ws, size_t vlen, cplx<T>* x, const cplx<T>* b, int nrhs, int m, double tol,
                 int max_cycles, bool final_residual, bool flexible, AOp A, MOp M, KrylovResult* res,
                 bool resume = false, const double* tol_rhs = nullptr, bool df = false) {
  // resume: x and ws.r already hold an iterate and its residual b - A x (continued
  // restart cycles); tol_rhs: one relative tolerance per right-hand side
  cudaStream_t st = h->st;
  const size_t rs = vlen;
  const size_t vs = (size_t)ws.batch * vlen;
  GmresState& gs = ws.gs;
  if (m > ws.m) fail(DDAMG_ERR_ARG, "Krylov length exceeds the workspace");
  GmresState s = gs;
  s.m = m;
  blas_norm2<T>(s.beta, b, vlen, nrhs, rs, st);
  CK(cudaMemcpyAsync(h->h_scal, s.beta, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
  sync(h);
  std::vector<double> bnorm(h->h_scal, h->h_scal + nrhs), target(nrhs);
  for (int r = 0; r < nrhs; ++r) target[r] = (tol_rhs ? tol_rhs[r] : tol) * bnorm[r];
  CK(cudaMemcpyAsync(s.target, target.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
  if (!resume) {
    blas_zero<T>(x, vlen, nrhs, rs, st);
    blas_convert<T, T>(ws.r, b, vlen, nrhs, rs, rs, st);
  } else {
    blas_norm2<T>(s.beta, ws.r, vlen, nrhs, rs, st);   // residual norms of the given iterates
  }
  if (res) {
    res->iterations.assign(nrhs, 0);
    res->cycles.assign(nrhs, 0);
    res->converged.assign(nrhs, 0);
    res->true_residual.assign(nrhs, 1.0);
  }
  std::vector<int> conv(nrhs, 0);
  for (int r = 0; r < nrhs; ++r) conv[r] = bnorm[r] == 0.0;
  for (int cycle = 0; cycle < max_cycles; ++cycle) {
    gmres_begin(s, nrhs, st);
    blas_scale_to<T>(ws.V, ws.r, s.inv, vlen, nrhs, rs, st);
    int kmax = 0;
    for (int j = 0; j < m; ++j) {
      cplx<T>* vj = ws.V + (size_t)j * vs;
      cplx<T>* zj = flexible ? ws.Z + (size_t)j * vs : vj;
      cplx<T>* w = ws.V + (size_t)(j + 1) * vs;
      if (flexible) M(zj, vj);
      A(w, zj, nullptr);
      {
        Prof pr(h, DDAMG_PROF_OUTER_ORTHO, (double)(2 * (j + 1) + 3) * 2 * vlen * nrhs * 2.0 * sizeof(T));
        bool done = false;
        if constexpr (sizeof(T) == 8) {
          if (df) {   // CGS2 in double-FP32 arithmetic on the FP64 basis
            blas_multidot_df(s.h1, m + 1, ws.V, vs, j + 1, w, vlen, nrhs, rs, st);
            blas_multiaxpy_df(w, ws.V, vs, j + 1, s.h1, m + 1, -1.0, vlen, nrhs, rs, st);
            blas_multidot_df(s.h2, m + 1, ws.V, vs, j + 1, w, vlen, nrhs, rs, st);
            blas_multiaxpy_df(w, ws.V, vs, j + 1, s.h2, m + 1, -1.0, vlen, nrhs, rs, st);
            done = true;
          }
        }
        if (!done) {
          blas_multidot<T>(s.h1, m + 1, ws.V, vs, j + 1, w, vlen, nrhs, rs, st);
          blas_multiaxpy<T>(w, ws.V, vs, j + 1, s.h1, m + 1, -1.0, vlen, nrhs, rs, st);
          blas_multidot<T>(s.h2, m + 1, ws.V, vs, j + 1, w, vlen, nrhs, rs, st);
          blas_multiaxpy<T>(w, ws.V, vs, j + 1, s.h2, m + 1, -1.0, vlen, nrhs, rs, st);
        }
        blas_norm2<T>(s.wnorm, w, vlen, nrhs, rs, st);
        gmres_step(s, j, nrhs, st);
        blas_scale_to<T>(w, w, s.inv, vlen, nrhs, rs, st);
      }
      kmax = j + 1;
      ws.host_steps += 1;
      CK(cudaMemcpyAsync(h->h_done, s.done, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st));
      sync(h);
      bool all = true;
      for (int r = 0; r < nrhs; ++r) all = all && h->h_done[r];
      if (all) break;
    }
    gmres_solve_y(s, nrhs, st);
    blas_multiaxpy<T>(x, flexible ? ws.Z : ws.V, vs, kmax, s.y, m, 1.0, vlen, nrhs, rs, st);
    if (res) {
      CK(cudaMemcpyAsync(h->h_kr, s.kr, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st));
      sync(h);
      for (int r = 0; r < nrhs; ++r)
        if (!conv[r]) {
          res->iterations[r] += h->h_kr[r];
          res->cycles[r] = cycle + 1;
        }
    }
    if (cycle == max_cycles - 1 && !final_residual) break;
    A(ws.r, x, b);   // r = b - A x
    blas_norm2<T>(s.beta, ws.r, vlen, nrhs, rs, st);
    CK(cudaMemcpyAsync(h->h_scal, s.beta, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    sync(h);
    bool all = true;
    for (int r = 0; r < nrhs; ++r) {
      const double beta = h->h_scal[r];
      if (res && !conv[r]) res->true_residual[r] = bnorm[r] > 0 ? beta / bnorm[r] : 0.0;
      if (beta <= target[r]) conv[r] = 1;
      all = all && conv[r];
    }
    if (all) break;
  }
  if (res)
    for (int r = 0; r < nrhs; ++r) {
      res->converged[r] = conv[r];
      if (bnorm[r] == 0.0) res->true_residual[r] = 0.0;
    }
}

// ---------------------------------------------------------------------------
// Device-driven (F)GMRES, emitted into a stream capture: the restart cycles and
// the Arnoldi steps are conditional WHILE nodes whose conditions are set by the
// kernels (k_kry_start / k_cycle_begin / k_arnoldi / k_cycle_end), so the
// solve needs no host round trip.  Same arithmetic and stopping rules as
// krylov_host.
cudaGraphConditionalHandle create_cond(ddamg_handle* h) {
  cudaStreamCaptureStatus status;
  cudaGraph_t g = nullptr;
  CK(cudaStreamGetCaptureInfo(h->st, &status, nullptr, &g, nullptr, nullptr, nullptr));
  if (status != cudaStreamCaptureStatusActive || !g) fail(DDAMG_ERR_CUDA, "conditional node outside a capture");
  cudaGraphConditionalHandle hc;
  CK(cudaGraphConditionalHandleCreate(&hc, g, 0, 0));
  return hc;
}

template <class F>
void emit_while(ddamg_handle* h, cudaGraphConditionalHandle hc, F body) {
  cudaStreamCaptureStatus status;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(h->st, &status, nullptr, &g, &deps, &ed, &nd));
  cudaGraphNodeParams prm = {};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = hc;
  prm.conditional.type = cudaGraphCondTypeWhile;
  prm.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps, ed, nd, &prm));
  CK(cudaStreamUpdateCaptureDependencies(h->st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaGraph_t bodyg = prm.conditional.phGraph_out[0];
  const int d = h->cap.depth + 1;
  if (d >= 12) fail(DDAMG_ERR_ARG, "conditional nesting too deep");
  cudaStream_t saved = h->st;
  h->cap.depth = d;
  h->st = h->cap.s[d];
  CK(cudaStreamBeginCaptureToGraph(h->st, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  body();
  cudaGraph_t out = nullptr;
  CK(cudaStreamEndCapture(h->st, &out));
  h->st = saved;
  h->cap.depth = d - 1;
}

template <typename T, class AOp, class MOp>
void krylov_dev(ddamg_handle* h, Work<T>& ws, size_t vlen, cplx<T>* x, const cplx<T>* b, int nrhs, int m, double tol,
                int max_cycles, bool flexible, AOp A, MOp M) {
  if (m > ws.m) fail(DDAMG_ERR_ARG, "Krylov length exceeds the workspace");
  const size_t vs = (size_t)ws.batch * vlen;
  GmresState s = ws.gs;
  s.m = m;
  blas_zero<T>(x, vlen, nrhs, vlen, h->st);
  blas_convert<T, T>(ws.r, b, vlen, nrhs, vlen, vlen, h->st);
  blas_norm2<T>(s.beta, b, vlen, nrhs, vlen, h->st);
  const cudaGraphConditionalHandle hcycle = create_cond(h);
  kry_start(s, nrhs, tol, hcycle, h->st);
  emit_while(h, hcycle, [&] {
    const cudaGraphConditionalHandle hinner = create_cond(h);
    kry_cycle_begin<T>(s, ws.V, ws.cur, ws.r, vlen, nrhs, hinner, h->st);
    emit_while(h, hinner, [&] {
      if (flexible) {
        M(ws.zc, ws.cur);
        A(ws.wv, ws.zc, nullptr);
      } else {
        A(ws.wv, ws.cur, nullptr);
      }
      CK(kry_arnoldi<T>(s, ws.V, vs, flexible ? ws.Z : nullptr, ws.zc, ws.wv, ws.cur, vlen, nrhs, hinner, h->st));
    });
    gmres_solve_y(s, nrhs, h->st);
    blas_multiaxpy<T>(x, flexible ? ws.Z : ws.V, vs, m, s.y, m, 1.0, vlen, nrhs, vlen, h->st);
    A(ws.r, x, b);
    blas_norm2<T>(s.beta, ws.r, vlen, nrhs, vlen, h->st);
    kry_cycle_end(s, nrhs, max_cycles, hcycle, h->st);
  });
}

// host-driven while eager, device-driven while capturing a graph
template <typename T, class AOp, class MOp>
void krylov(ddamg_handle* h, Work<T>& ws, size_t vlen, cplx<T>* x, const cplx<T>* b, int nrhs, int m, double tol,
            int max_cycles, bool final_residual, bool flexible, AOp A, MOp M, KrylovResult* res) {
  if (h->cap.active) krylov_dev<T>(h, ws, vlen, x, b, nrhs, m, tol, max_cycles, flexible, A, M);
  else krylov_host<T>(h, ws, vlen, x, b, nrhs, m, tol, max_cycles, final_residual, flexible, A, M, res);
}

// ---------------------------------------------------------------------------
// coarsest level: odd-even preconditioned GMRES (Sec. 3)
template <typename T>
const CoarsestPlan* cluster_plan(ddamg_handle* h) {
  if (!h->use_cluster) return nullptr;
  if (sizeof(T) == 4) return h->have_cplan32 ? &h->cplan32 : nullptr;
  return h->have_cplan64 ? &h->cplan64 : nullptr;
}

template <typename T>
void coarse_solve(ddamg_handle* h, cplx<T>* x, const cplx<T>* b, int nrhs) {
  Level& C = h->lv[h->L - 1];
  Work<T>& w = work<T>(C);
  CoarseOp<T>& op = cop<T>(C);
  const size_t rs = C.vlen;
  if (!C.eo) {
    // odd extents: plain GMRES on D_L (same length, cycles and tolerance)
    auto A = [&](cplx<T>* out, const cplx<T>* in, const cplx<T>* bb) { apply_D<T>(h, C, out, in, bb, nrhs); };
    auto none = [](cplx<T>*, const cplx<T>*) {};
    krylov<T>(h, w, C.vlen, x, b, nrhs, h->p.coarse_restart, h->p.coarse_tol, h->p.coarse_cycles, true, false, A,
              none, nullptr);
    return;
  }
  if (const CoarsestPlan* pl = cluster_plan<T>(h)) {
    // the whole odd-even GMRES in one cluster-resident kernel per right-hand side
    CK(coarsest_cluster_solve<T>(x, b, op, *pl, h->cgeo, nrhs, rs, h->p.coarse_restart, h->p.coarse_cycles,
                                 h->p.coarse_tol, w.gs.ctl + 3, h->st));
    return;
  }
  cplx<T>*t1 = w.t[0], *bh = w.t[3], *xe = w.t[4];
  // bhat_e = b_e - D_eo D_oo^{-1} b_o
  coarse_schur_odd<T>(t1, nullptr, b, op, 1.0, 0.0, nrhs, rs, h->st);
  coarse_schur_even<T>(bh, nullptr, t1, b, op, 1.0, 0.0, -1.0, nrhs, rs, h->st);
  // Dhat x_e = D_ee x_e - D_eo D_oo^{-1} D_oe x_e (residual form: b - Dhat x_e)
  auto schur = [&](cplx<T>* out, const cplx<T>* in, const cplx<T>* bb) {
    coarse_schur_odd<T>(t1, in, nullptr, op, 0.0, 1.0, nrhs, rs, h->st);
    if (bb) coarse_schur_even<T>(out, in, t1, bb, op, 1.0, -1.0, 1.0, nrhs, rs, h->st);
    else coarse_schur_even<T>(out, in, t1, nullptr, op, 0.0, 1.0, -1.0, nrhs, rs, h->st);
  };
  auto none = [](cplx<T>*, const cplx<T>*) {};
  krylov<T>(h, w, C.vlen, xe, bh, nrhs, h->p.coarse_restart, h->p.coarse_tol, h->p.coarse_cycles, true, false, schur,
            none, nullptr);
  // z_e = x_e;  z_o = D_oo^{-1} (b_o - D_oe x_e)
  blas_convert<T, T>(x, xe, rs, nrhs, rs, rs, h->st);
  coarse_schur_odd<T>(x, xe, b, op, 1.0, -1.0, nrhs, rs, h->st);
}

// one K-cycle from level l (Alg. 2): z = K(l, b)
template <typename T>
void kcycle(ddamg_handle* h, int l, cplx<T>* z, const cplx<T>* b, int nrhs) {
  Level& F = h->lv[l];
  Level& C = h->lv[l + 1];
  Work<T>& wc = work<T>(C);
  blas_zero<T>(z, F.vlen, nrhs, F.vlen, h->st);
  if (h->p.mu > 0) {
    sap<T>(h, F, z, b, nrhs, h->p.mu);
    cplx<T>* r = work<T>(F).r;
    apply_D<T>(h, F, r, z, b, nrhs);
    restrict_lv<T>(h, l, wc.bc, r, nrhs);
  } else {
    restrict_lv<T>(h, l, wc.bc, b, nrhs);
  }
  if (l + 1 == h->L - 1) {
    coarse_solve<T>(h, wc.xs, wc.bc, nrhs);
  } else {
    auto A = [&](cplx<T>* out, const cplx<T>* in, const cplx<T>* bb) { apply_D<T>(h, C, out, in, bb, nrhs); };
    auto M = [&](cplx<T>* out, const cplx<T>* in) { kcycle<T>(h, l + 1, out, in, nrhs); };
    krylov<T>(h, wc, C.vlen, wc.xs, wc.bc, nrhs, h->p.kcycle_len, h->p.kcycle_tol, h->p.kcycle_cycles, false, true,
              A, M, nullptr);
  }
  prolong_lv<T>(h, l, z, wc.xs, nrhs, h->p.mu > 0);
  sap<T>(h, F, z, b, nrhs, h->p.nu);
}

// ---------------------------------------------------------------------------
// CUDA graphs of whole K-cycles, one per (start level, precision, batch size,
// profiling mask); captured on first use, replayed afterwards.  The graph reads
// its right-hand side from Work.gin of the start level and writes Work.gout.
template <typename T>
GraphEntry* get_graph(ddamg_handle* h, int l0, int nrhs) {
  for (GraphEntry* e : h->graphs)
    if (e->l0 == l0 && e->tsize == (int)sizeof(T) && e->nrhs == nrhs && e->prof == h->prof) return e;
  GraphEntry* e = new GraphEntry();
  e->l0 = l0;
  e->tsize = (int)sizeof(T);
  e->nrhs = nrhs;
  e->prof = h->prof;
  Work<T>& w = work<T>(h->lv[l0]);
  cudaStream_t saved = h->st;
  sync(h);
  h->cap.active = true;
  h->cap.depth = 0;
  h->capturing = e;
  h->st = h->cap.s[0];
  cudaGraph_t graph = nullptr;
  try {
    CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed));
    kcycle<T>(h, l0, w.gout, w.gin, nrhs);
    CK(cudaStreamEndCapture(h->st, &graph));
  } catch (...) {
    cudaGraph_t junk = nullptr;
    cudaStreamEndCapture(h->cap.s[0], &junk);
    if (junk) cudaGraphDestroy(junk);
    cudaGetLastError();
    h->st = saved;
    h->cap.active = false;
    h->capturing = nullptr;
    for (cudaEvent_t ev : e->ev) cudaEventDestroy(ev);
    delete e;
    throw;
  }
  h->st = saved;
  h->cap.active = false;
  h->cap.depth = 0;
  h->capturing = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&e->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    for (cudaEvent_t ev : e->ev) cudaEventDestroy(ev);
    delete e;
    fail(DDAMG_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
  }
  h->graphs.push_back(e);
  return e;
}

// z = K-cycle(l0, b) through the captured graph (or eagerly when graphs are off)
template <typename T>
void kcycle_run(ddamg_handle* h, int l0, cplx<T>* z, const cplx<T>* b, int nrhs) {
  if (!h->use_graphs) {
    kcycle<T>(h, l0, z, b, nrhs);
    return;
  }
  GraphEntry* e = get_graph<T>(h, l0, nrhs);
  Work<T>& w = work<T>(h->lv[l0]);
  const size_t vl = h->lv[l0].vlen;
  blas_convert<T, T>(w.gin, b, vl, nrhs, vl, vl, h->st);
  count_launch(1);
  CK(cudaGraphLaunch(e->exec, h->st));
  blas_convert<T, T>(z, w.gout, vl, nrhs, vl, vl, h->st);
  if (!e->ev.empty()) {
    sync(h);
    for (size_t q = 0; q < e->ev_kind.size(); ++q) {
      float t = 0;
      CK(cudaEventElapsedTime(&t, e->ev[2 * q], e->ev[2 * q + 1]));
      h->prof_graph_ms[e->ev_kind[q]] += t;
      h->prof_count[e->ev_kind[q]] += 1;
      h->prof_bytes[e->ev_kind[q]] += e->ev_bytes[q];
    }
  }
}

void free_graphs(ddamg_handle* h) {
  for (GraphEntry* e : h->graphs) {
    if (e->exec) cudaGraphExecDestroy(e->exec);
    for (cudaEvent_t ev : e->ev) cudaEventDestroy(ev);
    delete e;
  }
  h->graphs.clear();
}

// ---------------------------------------------------------------------------
// hierarchy construction
// allow_loose: aggregates and SAP blocks need not nest (coarse levels); the sites are
// then ordered by aggregate and the SAP blocks are addressed through site tables
void make_geom(Geom& g, const int L[4], const int A[4], const int B[4], bool allow_loose = false) {
  bool b_in_a = true, a_in_b = true;
  for (int d = 0; d < 4; ++d) {
    if (L[d] <= 0 || A[d] <= 0 || B[d] <= 0 || L[d] % A[d] || L[d] % B[d])
      fail(DDAMG_ERR_ARG, "lattice extent " + std::to_string(L[d]) + " is not tiled by aggregate " +
                              std::to_string(A[d]) + " and SAP block " + std::to_string(B[d]) + " in direction " +
                              std::to_string(d));
    b_in_a = b_in_a && (A[d] % B[d] == 0);
    a_in_b = a_in_b && (B[d] % A[d] == 0);
  }
  const bool nest = b_in_a || a_in_b;
  if (!nest && !allow_loose)
    fail(DDAMG_ERR_ARG, "on the fine level aggregates and SAP blocks must nest (one must tile the other)");
  const int* O = nest ? (b_in_a ? A : B) : A;
  const int* I = nest ? (b_in_a ? B : A) : A;
  g.V = g.vA = g.vB = g.vI = g.nIO = g.nAgg = 1;
  for (int d = 0; d < 4; ++d) {
    g.L[d] = L[d];
    g.A[d] = A[d];
    g.B[d] = B[d];
    g.O[d] = O[d];
    g.I[d] = I[d];
    g.nO[d] = L[d] / O[d];
    g.nI[d] = O[d] / I[d];
    g.V *= L[d];
    g.vA *= A[d];
    g.vB *= B[d];
    g.vI *= I[d];
    g.nIO *= g.nI[d];
    g.nAgg *= L[d] / A[d];
  }
  g.nBlk = g.V / g.vB;
}

void build_block_lists(ddamg_handle* h, Level& L) {
  const Geom& g = L.g;
  for (int d = 0; d < 4; ++d) {
    const int nb = g.L[d] / g.B[d];
    if (nb != 1 && nb % 2)
      fail(DDAMG_ERR_ARG, "red-black SAP needs an even number of blocks per direction on level " +
                              std::to_string(L.idx));
  }
  if (L.fine ? g.vB > 1024 : g.vB * L.n > 4 * 1024)
    fail(DDAMG_ERR_ARG, "SAP block too large on level " + std::to_string(L.idx));
  std::vector<int> lists[2];
  if (L.fine) {   // fine level: SAP blocks are contiguous index ranges
    for (int b = 0; b < g.nBlk; ++b) {
      int c[4];
      geom_coords(g, b * g.vB, c);
      lists[geom_block_colour(g, c)].push_back(b);
    }
  } else {        // coarse levels: blocks in lexicographic order, their sites through tables
    int nb[4];
    for (int d = 0; d < 4; ++d) nb[d] = g.L[d] / g.B[d];
    std::vector<int> bsite((size_t)g.nBlk * g.vB), bloc(g.V);
    for (int b = 0; b < g.nBlk; ++b) {
      int bc[4], c[4], lc[4];
      delin4(b, nb, bc);
      for (int loc = 0; loc < g.vB; ++loc) {
        delin4(loc, g.B, lc);
        for (int d = 0; d < 4; ++d) c[d] = bc[d] * g.B[d] + lc[d];
        const int site = geom_index(g, c);
        bsite[(size_t)b * g.vB + loc] = site;
        bloc[site] = loc;
      }
      for (int d = 0; d < 4; ++d) c[d] = bc[d] * g.B[d];
      lists[geom_block_colour(g, c)].push_back(b);
    }
    L.bsite = dalloc<int>(h, bsite.size());
    L.bloc = dalloc<int>(h, bloc.size());
    CK(cudaMemcpy(L.bsite, bsite.data(), sizeof(int) * bsite.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.bloc, bloc.data(), sizeof(int) * bloc.size(), cudaMemcpyHostToDevice));
    L.c64.bsite = L.c32.bsite = L.bsite;
    L.c64.bloc = L.c32.bloc = L.bloc;
    L.sap_gcnt = dalloc<unsigned>(h, 1);
  }
  for (int c = 0; c < 2; ++c) {
    L.nblocks[c] = (int)lists[c].size();
    L.blocks[c] = dalloc<int>(h, lists[c].size());
    if (!lists[c].empty())
      CK(cudaMemcpy(L.blocks[c], lists[c].data(), sizeof(int) * lists[c].size(), cudaMemcpyHostToDevice));
  }
}

// Workspaces by role: the fine level only needs the residual of the pre-smoother
// and the fixed input/output of a captured K-cycle; the outer FGMRES only its
// bases and residual; coarse levels the inner (F)GMRES and the restricted
// right-hand side / coarse iterate; the coarsest also the odd-even temporaries.
enum WorkRole { WORK_FINE, WORK_COARSE, WORK_COARSEST, WORK_OUTER };

template <typename T>
void alloc_work(ddamg_handle* h, Level& L, Work<T>& w, int m, WorkRole role, int batch) {
  const size_t vl = L.vlen * (size_t)batch;
  const bool flexible = role != WORK_COARSEST;
  w.m = m;
  w.batch = batch;
  w.r = dalloc<cplx<T>>(h, vl);
  if (role != WORK_OUTER) {
    w.gin = dalloc<cplx<T>>(h, vl);
    w.gout = dalloc<cplx<T>>(h, vl);
  }
  if (role == WORK_COARSE || role == WORK_COARSEST) {
    w.bc = dalloc<cplx<T>>(h, vl);
    w.xs = dalloc<cplx<T>>(h, vl);
    w.cur = dalloc<cplx<T>>(h, vl);
    w.zc = dalloc<cplx<T>>(h, vl);
    w.wv = dalloc<cplx<T>>(h, vl);
  }
  if (role == WORK_COARSEST)
    for (int k = 0; k < 5; ++k) w.t[k] = dalloc<cplx<T>>(h, vl);
  if (m > 0) {
    w.V = dalloc<cplx<T>>(h, vl * (m + 1));
    if (flexible) w.Z = dalloc<cplx<T>>(h, vl * m);
  }
  GmresState& s = w.gs;
  const int mm = m > 0 ? m : 1;
  s.m = mm;
  s.H = dalloc<cplx<double>>(h, (size_t)batch * (mm + 1) * mm);
  s.cs = dalloc<double>(h, (size_t)batch * mm);
  s.sn = dalloc<cplx<double>>(h, (size_t)batch * mm);
  s.g = dalloc<cplx<double>>(h, (size_t)batch * (mm + 1));
  s.h1 = dalloc<cplx<double>>(h, (size_t)batch * (mm + 1));
  s.h2 = dalloc<cplx<double>>(h, (size_t)batch * (mm + 1));
  s.y = dalloc<cplx<double>>(h, (size_t)batch * mm);
  s.wnorm = dalloc<double>(h, batch);
  s.inv = dalloc<double>(h, batch);
  s.beta = dalloc<double>(h, batch);
  s.target = dalloc<double>(h, batch);
  s.est = dalloc<double>(h, batch);
  s.done = dalloc<int>(h, batch);
  s.kr = dalloc<int>(h, batch);
  s.conv = dalloc<int>(h, batch);
  s.iters = dalloc<int>(h, batch);
  s.bnorm = dalloc<double>(h, batch);
  s.ctl = dalloc<int>(h, 4);
  CK(cudaMemset(s.ctl, 0, sizeof(int) * 4));
}

void gamma_products(double* out /* [6][4][4][2] */) {
  // chiral basis: gamma_t = [[0,1],[1,0]], gamma_k = [[0,-i s_k],[i s_k,0]]; mu = (t, z, y, x)
  typedef double c2[2];
  c2 gam[4][4][4];
  memset(gam, 0, sizeof(gam));
  const double sig[3][2][2][2] = {
      {{{0, 0}, {1, 0}}, {{1, 0}, {0, 0}}},     // sigma_x
      {{{0, 0}, {0, -1}}, {{0, 1}, {0, 0}}},    // sigma_y
      {{{1, 0}, {0, 0}}, {{0, 0}, {-1, 0}}}};   // sigma_z
  for (int i = 0; i < 2; ++i) {
    gam[0][i][2 + i][0] = 1;
    gam[0][2 + i][i][0] = 1;
  }
  const int which[4] = {-1, 2, 1, 0};   // mu = z, y, x use sigma_z, sigma_y, sigma_x
  for (int mu = 1; mu < 4; ++mu) {
    const int k = which[mu];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        const double re = sig[k][i][j][0], im = sig[k][i][j][1];
        // upper right block: -i sigma = (im, -re) ; lower left: i sigma = (-im, re)
        gam[mu][i][2 + j][0] = im;
        gam[mu][i][2 + j][1] = -re;
        gam[mu][2 + i][j][0] = -im;
        gam[mu][2 + i][j][1] = re;
      }
  }
  int p = 0;
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = mu + 1; nu < 4; ++nu, ++p)
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
          double re = 0, im = 0;
          for (int k = 0; k < 4; ++k) {
            const double ar = gam[mu][i][k][0], ai = gam[mu][i][k][1];
            const double br = gam[nu][k][j][0], bi = gam[nu][k][j][1];
            re += ar * br - ai * bi;
            im += ar * bi + ai * br;
          }
          out[((p * 4 + i) * 4 + j) * 2 + 0] = re;
          out[((p * 4 + i) * 4 + j) * 2 + 1] = im;
        }
}

void check_err_flag(ddamg_handle* h, const char* what) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  sync(h);
  if (e) {
    CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->st));
    sync(h);
    fail(DDAMG_ERR_SINGULAR, what);
  }
}

// FP16 storage copies: allocated on first use, filled from the FP64 data after
// every change of it, and read by the FP32 kernels while h->half is set.
void half_alloc(ddamg_handle* h) {
  for (int l = 0; l < h->L; ++l) {
    Level& L = h->lv[l];
    if (L.fine && !L.Uh) {
      L.Uh = dalloc<__half2>(h, (size_t)36 * L.g.V);
      L.clovh = dalloc<__half2>(h, (size_t)36 * L.g.V);
    }
    if (!L.fine && !L.blkh) {
      L.blkh = dalloc<__half2>(h, (size_t)L.g.V * 9 * L.n * L.n);
      L.bscale = dalloc<float>(h, (size_t)L.g.V);
    }
    if (!L.coarsest && !L.Ph) {
      L.Ph = dalloc<__half2>(h, L.vlen * (size_t)L.N);
      L.pscale = dalloc<float>(h, (size_t)L.g.nAgg * 2);
    }
  }
}

// double-FP32 copies of the fine links and clover term (allocated on first use)
void df_refresh(ddamg_handle* h) {
  Level& F = h->lv[0];
  if (!F.Udf) {
    F.Udf = dalloc<cplx<dfl>>(h, (size_t)36 * F.g.V);
    F.clovdf = dalloc<dfl>(h, (size_t)72 * F.g.V);
  }
  double_to_df(reinterpret_cast<dfl*>(F.Udf), reinterpret_cast<const double*>(F.f64.U), (size_t)72 * F.g.V, h->st);
  double_to_df(F.clovdf, F.f64.clov, (size_t)72 * F.g.V, h->st);
}

void half_refresh_fine(ddamg_handle* h) {
  Level& F = h->lv[0];
  links_to_half(F.Uh, F.f64.U, (size_t)36 * F.g.V, h->st);
  clover_to_half(F.clovh, F.f64.clov, F.g.V, h->m0 + 4.0, h->st);
}

// P_l and D_{l+1}
void half_refresh(ddamg_handle* h, int l) {
  Level& F = h->lv[l];
  Level& C = h->lv[l + 1];
  p_to_half(F.Ph, F.pscale, F.P64, F.g, F.fine, F.n, F.N, h->st);
  blocks_to_half(C.blkh, C.bscale, C.c64.blk, C.g.V, C.n, h->st);
}

void half_bind(ddamg_handle* h) {
  for (auto& L : h->lv) {
    if (L.fine) {
      L.f32.Uh = h->half ? L.Uh : nullptr;
      L.f32.clovh = h->half ? L.clovh : nullptr;
      L.f32.shift = (float)(h->m0 + 4.0);
    } else {
      L.c32.blkh = h->half ? L.blkh : nullptr;
      L.c32.bscale = h->half ? L.bscale : nullptr;
    }
  }
}

// Schur SAP tables of the fine level: A(x)^{-1} per site in FP64 (temporary), then the tables with
// the clover term on even and the inverse on odd sites, in FP32 and FP16.  A zero pivot is an error.
void schur_tables(ddamg_handle* h) {
  Level& F = h->lv[0];
  if (!F.mix32) F.mix32 = dalloc<float>(h, (size_t)72 * F.g.V);
  if (!F.mixh) F.mixh = dalloc<__half2>(h, (size_t)36 * F.g.V);
  double* inv = nullptr;
  if (cudaMalloc(&inv, sizeof(double) * 72 * (size_t)F.g.V) != cudaSuccess) {
    cudaGetLastError();
    fail(DDAMG_ERR_OOM, "temporary for the clover inverse");
  }
  clover_inverse(inv, F.f64.clov, F.g.V, h->d_err, h->st);
  clover_mix(F.mix32, F.mixh, F.f64.clov, inv, F.g, h->m0 + 4.0, h->st);
  const cudaError_t e = cudaStreamSynchronize(h->st);
  cudaFree(inv);
  CK(e);
  check_err_flag(h, "singular site-diagonal block (clover inverse)");
}

// the 4^4 Schur kernel's conditions: FP32 preconditioner, fine SAP blocks 4^4 and the inner tile
void schur_check(ddamg_handle* h) {
  const Geom& g = h->lv[0].g;
  for (int d = 0; d < 4; ++d)
    if (g.B[d] != 4 || g.I[d] != 4)
      fail(DDAMG_ERR_ARG, "Schur SAP block solves need 4^4 fine SAP blocks that tile the aggregates");
}

void schur_bind(ddamg_handle* h) {
  Level& F = h->lv[0];
  F.f32.schur = h->sap_schur;
  F.f32.mix32 = h->sap_schur ? F.mix32 : nullptr;
  F.f32.mixh = h->sap_schur && h->half ? F.mixh : nullptr;
}

// the fine operator from a gauge field in the ABI layout: links (FP64, FP32), the clover term
// with the mass shift (FP64, FP32)
void import_operator(ddamg_handle* h, const double* gauge) {
  Level& F = h->lv[0];
  const size_t gbytes = sizeof(cplx<double>) * 36 * (size_t)F.g.V;
  const cplx<double>* gd = static_cast<const cplx<double>*>(dev_in(h, gauge, gbytes, 0));
  links_import<double>(F.f64.U, gd, F.g, h->st);
  links_import<float>(F.f32.U, gd, F.g, h->st);
  clover_build(F.f64.clov, gd, F.g, h->m0, h->csw, h->st);
  real_convert<float>(F.f32.clov, F.f64.clov, (size_t)72 * F.g.V, h->st);
}

// Autotuner of the kernels that read FP16 operator data for a whole batch: on every level, time
// each candidate kernel for one application of the handle's batch size (after a warm-up, CUDA
// events on the library stream) and keep the fastest:
//   coarse stencil (levels >= 1): CUDA-core kernel (0), tensor cores with k-split 1..4;
//   restriction l -> l+1: per-right-hand-side kernel (0), tensor cores with k-split 1..4;
//   prolongation l+1 -> l: per-right-hand-side kernel (0), one CTA per aggregate for the batch (1).
// The choice is made once per level and used for every batch size, so a right-hand side keeps the
// same bits alone and inside a batch.  Timing does not depend on the operand values.
template <class Run>
int time_candidates(ddamg_handle* h, double* ms_out, int ncand, Run run) {
  // two interleaved rounds (clocks and caches settle over the first), minimum per candidate
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int k = 0; k < ncand; ++k) ms_out[k] = -1.0;
  for (int round = 0; round < 2; ++round)
    for (int k = 0; k < ncand; ++k) {
      if (!run(k, true)) continue;   // warm-up; false: the candidate does not fit
      run(k, true);
      constexpr int reps = 10;
      CK(cudaEventRecord(e0, h->st));
      for (int q = 0; q < reps; ++q) run(k, false);
      CK(cudaEventRecord(e1, h->st));
      CK(cudaEventSynchronize(e1));
      CK(cudaGetLastError());
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      const double t = ms / reps;
      if (ms_out[k] < 0 || t < ms_out[k]) ms_out[k] = t;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int best = 0;
  for (int k = 1; k < ncand; ++k)
    if (ms_out[k] >= 0 && ms_out[k] < ms_out[best]) best = k;
  return best;
}

// Whether the persistent SAP launch of level L runs on this device: one eager call and one call
// from an instantiated graph (cooperative cluster launches in stream capture), both without error
// and without a barrier time-out.
bool persist_works(ddamg_handle* h, Level& L) {
  Work<float>& w = work<float>(L);
  const int mr = h->p.mr_steps;
  sync(h);
  bool ok = coarse_sap_persist(w.gout, w.gin, L.c32, L.blocks[0], L.nblocks[0], L.blocks[1], L.nblocks[1], 1, L.vlen,
                               mr, 1, L.sap_nbpc, L.sap_gcnt, h->st) == cudaSuccess;
  cudaGetLastError();
  sync(h);
  int e = 0;
  CK(cudaMemcpy(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    CK(cudaMemset(h->d_err, 0, sizeof(int)));
    ok = false;
  }
  if (!ok) return false;
  cudaStream_t s = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    const cudaError_t e1 = coarse_sap_persist(w.gout, w.gin, L.c32, L.blocks[0], L.nblocks[0], L.blocks[1],
                                              L.nblocks[1], 1, L.vlen, mr, 1, L.sap_nbpc, L.sap_gcnt, s);
    const cudaError_t e2 = cudaStreamEndCapture(s, &g);
    ok = e1 == cudaSuccess && e2 == cudaSuccess && g != nullptr;
  }
  if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
  if (ok) ok = cudaGraphLaunch(ge, s) == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess;
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(s);
  cudaGetLastError();
  CK(cudaMemcpy(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    CK(cudaMemset(h->d_err, 0, sizeof(int)));
    ok = false;
  }
  return ok;
}

void tune_kernels(ddamg_handle* h) {
  const int B = h->max_batch;
  for (int l = 0; l < h->L; ++l) {
    Level& L = h->lv[l];
    for (int t = 0; t < 4; ++t)
      for (int k = 0; k < 5; ++k) h->tune_ms[t][l][k] = -1.0;
    L.c32.tc_ks = 0;
    L.tr_ks = 0;
    L.pr_batch = 0;
    L.sap_persist = 0;
    if (!h->half) continue;
    // coarse SAP: one launch per colour sweep (0) or one persistent launch per smoother call (1);
    // entries 2..4 of the record: clusters of the persistent launch's shape the device holds at
    // once, clusters the level needs, SAP blocks of each colour per cluster (0: no shape fits)
    int maxcl = -1;
    L.sap_nbpc = 0;
    const bool pfits = !L.fine && !L.coarsest && h->persist_force != 0 &&
                       coarse_sap_persist_fits(L.c32, L.nblocks[0], L.nblocks[1], &maxcl, &L.sap_nbpc,
                                               h->persist_force == 2 ? 2 : 1);
    if (!L.fine && !L.coarsest) {
      const int nb = L.nblocks[0] > L.nblocks[1] ? L.nblocks[0] : L.nblocks[1];
      h->tune_ms[DDAMG_TUNE_SAP][l][2] = maxcl;
      h->tune_ms[DDAMG_TUNE_SAP][l][3] = pfits ? (nb + L.sap_nbpc - 1) / L.sap_nbpc : nb;
      h->tune_ms[DDAMG_TUNE_SAP][l][4] = L.sap_nbpc;
    }
    if (pfits && persist_works(h, L)) {
      if (h->persist_force >= 1) {
        L.sap_persist = 1;
      } else {
        Work<float>& w = work<float>(L);
        blas_zero<float>(w.gin, L.vlen, B, L.vlen, h->st);
        blas_zero<float>(w.gout, L.vlen, B, L.vlen, h->st);
        L.sap_persist = time_candidates(h, h->tune_ms[DDAMG_TUNE_SAP][l], 2, [&](int k, bool) {
          L.sap_persist = k;
          sap<float>(h, L, w.gout, w.gin, B, h->p.nu);
          return true;
        });
      }
    }
    if (h->tc_force >= 0) {
      const int f = h->tc_force;
      if (!L.fine) L.c32.tc_ks = (f > 0 && coarse_tc_fits(L.n, f)) ? f : 0;
      if (!L.coarsest) {
        L.tr_ks = (f > 0 && restrict_tc_fits(L.N, f)) ? f : 0;
        L.pr_batch = f > 0 ? 1 : 0;
      }
      continue;
    }
    Work<float>& w = work<float>(L);
    blas_zero<float>(w.gin, L.vlen, B, L.vlen, h->st);
    if (!L.fine) {
      CoarseOp<float>& op = L.c32;
      op.tc_ks = time_candidates(h, h->tune_ms[DDAMG_TUNE_COARSE][l], 5, [&](int k, bool) {
        if (k > 0 && !coarse_tc_fits(L.n, k)) return false;
        op.tc_ks = k;
        coarse_apply<float>(w.gout, w.gin, nullptr, op, B, L.vlen, SEL_FULL, 0, -1, h->st);
        return true;
      });
    }
    if (!L.coarsest) {
      Level& C = h->lv[l + 1];
      Work<float>& wc = work<float>(C);
      L.tr_ks = time_candidates(h, h->tune_ms[DDAMG_TUNE_RESTRICT][l], 5, [&](int k, bool) {
        if (k > 0 && !restrict_tc_fits(L.N, k)) return false;
        restrict_op<float>(wc.bc, w.gin, L.P32, L.g, C.g, L.fine, L.n, L.N, B, L.vlen, C.vlen, C.n, h->st, L.Ph,
                           L.pscale, k);
        return true;
      });
      blas_zero<float>(wc.bc, C.vlen, B, C.vlen, h->st);
      L.pr_batch = time_candidates(h, h->tune_ms[DDAMG_TUNE_PROLONG][l], 2, [&](int k, bool) {
        prolong_op<float>(w.gout, wc.bc, L.P32, L.g, C.g, L.fine, L.n, L.N, B, L.vlen, C.vlen, false, h->st, L.Ph,
                          L.pscale, k);
        return true;
      });
    }
  }
}

constexpr int SETUP_CHUNK = 4;   // columns / test vectors per pass of the setup's batched operations

// P_l from the test vectors, D_{l+1} = P_l^+ D_l P_l (FP64), FP32 copies, coarsest self inverses
// adds the wall-clock time of its scope to h->setup_s[l][kind] (the phases end with a sync)
struct SetupTimer {
  ddamg_handle* h;
  int l, kind;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  ~SetupTimer() {
    h->setup_s[l][kind] += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

void rebuild(ddamg_handle* h, int l) {
  SetupTimer tm{h, l, DDAMG_SETUP_REBUILD};
  Level& F = h->lv[l];
  Level& C = h->lv[l + 1];
  cudaStream_t st = h->st;
  const size_t tot = F.vlen * (size_t)F.N;
  blas_convert<double, double>(F.P64, F.tv64, tot, 1, 0, 0, st);
  orthonormalise(F.P64, F.g, F.fine, F.n, F.N, h->d_err, st);
  check_err_flag(h, "test vectors are linearly dependent on an aggregate");
  blas_convert<float, double>(F.P32, F.P64, tot, 1, 0, 0, st);
  // Galerkin: column (s', j) of every block = P^+ (term of D applied to P_j restricted to chirality s'),
  // in chunks of SETUP_CHUNK columns (bounded scratch).  A handle with the FP32 preconditioner forms
  // the product in FP32 from the FP32 copies of the operator and P (the preconditioner's setup runs
  // in single precision, Sec. 3); an FP64 handle in FP64.
  const int jb_max = F.N < SETUP_CHUNK ? F.N : SETUP_CHUNK;
  const int nc = C.n;
  const size_t nb = (size_t)C.g.V * 9 * nc * nc;
  if (h->p.precision != 0) {
    cplx<float>* tmp = static_cast<cplx<float>*>(scratch(h, 4, sizeof(cplx<float>) * F.vlen * jb_max));
    FineOp<float> fo = F.f32;   // FP32 storage, not the FP16 copies
    fo.Uh = nullptr;
    fo.clovh = nullptr;
    CoarseOp<float> co = F.c32;
    co.blkh = nullptr;
    co.bscale = nullptr;
    for (int sp = 0; sp < 2; ++sp)
      for (int k = 0; k < 9; ++k) {
        const int sel = k == 0 ? SEL_AGG_SELF : (k <= 4 ? SEL_AGG_FWD : SEL_AGG_BWD);
        const int mu = k == 0 ? 0 : (k - 1) % 4;
        for (int j0 = 0; j0 < F.N; j0 += jb_max) {
          const int jb = F.N - j0 < jb_max ? F.N - j0 : jb_max;
          const cplx<float>* pj = F.P32 + (size_t)j0 * F.vlen;
          if (F.fine) fine_dslash<float>(tmp, pj, nullptr, fo, jb, F.vlen, sel, mu, sp, st);
          else coarse_apply<float>(tmp, pj, nullptr, co, jb, F.vlen, sel, mu, sp, st);
          restrict_op<float>(C.c32.blk + (size_t)k * nc * nc + (size_t)(sp * F.N + j0) * nc, tmp, F.P32, F.g, C.g,
                             F.fine, F.n, F.N, jb, F.vlen, (size_t)nc, (size_t)9 * nc * nc, st);
        }
      }
    blas_convert<double, float>(C.c64.blk, C.c32.blk, nb, 1, 0, 0, st);
  } else {
    cplx<double>* tmp = static_cast<cplx<double>*>(scratch(h, 4, sizeof(cplx<double>) * F.vlen * jb_max));
    for (int sp = 0; sp < 2; ++sp)
      for (int k = 0; k < 9; ++k) {
        const int sel = k == 0 ? SEL_AGG_SELF : (k <= 4 ? SEL_AGG_FWD : SEL_AGG_BWD);
        const int mu = k == 0 ? 0 : (k - 1) % 4;
        for (int j0 = 0; j0 < F.N; j0 += jb_max) {
          const int jb = F.N - j0 < jb_max ? F.N - j0 : jb_max;
          apply_D<double>(h, F, tmp, F.P64 + (size_t)j0 * F.vlen, nullptr, jb, sel, mu, sp);
          restrict_op<double>(C.c64.blk + (size_t)k * nc * nc + (size_t)(sp * F.N + j0) * nc, tmp, F.P64, F.g, C.g,
                              F.fine, F.n, F.N, jb, F.vlen, (size_t)nc, (size_t)9 * nc * nc, st);
        }
      }
    blas_convert<float, double>(C.c32.blk, C.c64.blk, nb, 1, 0, 0, st);
  }
  if (C.coarsest && C.eo) {
    coarse_selfinv_build(C.c64.selfinv, C.c64.blk, C.g.V, nc, h->d_err, st);
    check_err_flag(h, "singular self block on the coarsest level");
    blas_convert<float, double>(C.c32.selfinv, C.c64.selfinv, (size_t)C.g.V * nc * nc, 1, 0, 0, st);
  }
  if (F.Ph) half_refresh(h, l);
  sync(h);
}

template <typename T>
void setup_smooth(ddamg_handle* h, int l) {
  SetupTimer tm{h, l, DDAMG_SETUP_SMOOTH};
  // the test vectors in chunks of SETUP_CHUNK (bounded scratch; each vector is smoothed on its own)
  Level& L = h->lv[l];
  const int jb_max = L.N < SETUP_CHUNK ? L.N : SETUP_CHUNK;
  cplx<T>* bT = static_cast<cplx<T>*>(scratch(h, 5, sizeof(cplx<T>) * L.vlen * jb_max));
  cplx<T>* xT = static_cast<cplx<T>*>(scratch(h, 6, sizeof(cplx<T>) * L.vlen * jb_max));
  for (int eta = 1; eta <= h->p.eta_passes; ++eta)
    for (int j0 = 0; j0 < L.N; j0 += jb_max) {
      const int jb = L.N - j0 < jb_max ? L.N - j0 : jb_max;
      const size_t tot = L.vlen * (size_t)jb;
      cplx<double>* tv = L.tv64 + (size_t)j0 * L.vlen;
      blas_convert<T, double>(bT, tv, tot, 1, 0, 0, h->st);
      blas_zero<T>(xT, tot, 1, 0, h->st);
      sap<T>(h, L, xT, bT, jb, eta);
      blas_convert<double, T>(tv, xT, tot, 1, 0, 0, h->st);
    }
  sync(h);
}

// host fields -> device level layout, SETUP_CHUNK fields at a time through the staging
// buffer (which stays allocated with the handle: chunks keep it near the gauge field's size)
void import_fields(ddamg_handle* h, Level& L, cplx<double>* dst, const double* src, int n) {
  for (int j0 = 0; j0 < n; j0 += SETUP_CHUNK) {
    const int jb = n - j0 < SETUP_CHUNK ? n - j0 : SETUP_CHUNK;
    const size_t bytes = sizeof(cplx<double>) * L.vlen * jb;
    const cplx<double>* d =
        static_cast<const cplx<double>*>(dev_in(h, src + (size_t)j0 * L.vlen * 2, bytes, 0));
    if (L.fine) fine_import<double>(dst + (size_t)j0 * L.vlen, d, L.g, jb, L.vlen, h->st);
    else coarse_import<double>(dst + (size_t)j0 * L.vlen, d, L.g, L.n, jb, L.vlen, h->st);
  }
}

// Alg. 3 on level l and below.  tv_random = NULL: the random start vectors are drawn on the
// device from params.seed (level 0: fields 0..N_0-1; level l: the fields beyond those that
// restriction provides); otherwise they are the caller's host or device fields.
void initial_setup_phase(ddamg_handle* h, int l, const double* const* tv_random) {
  Level& L = h->lv[l];
  if (l == 0) {
    if (!tv_random) {
      draw_fields(L.tv64, L.g, true, L.n, L.N, 0, 0, h->p.seed, L.vlen, h->st);
    } else {
      if (!tv_random[0]) fail(DDAMG_ERR_ARG, "random test vectors of level 0 missing");
      import_fields(h, L, L.tv64, tv_random[0], L.N);
    }
  } else {
    Level& U = h->lv[l - 1];
    const int take = L.N < U.N ? L.N : U.N;
    restrict_op<double>(L.tv64, U.tv64, U.P64, U.g, L.g, U.fine, U.n, U.N, take, U.vlen, L.vlen, L.n, h->st);
    if (L.N > take) {
      if (!tv_random) {
        draw_fields(L.tv64 + (size_t)take * L.vlen, L.g, false, L.n, L.N - take, 0, l, h->p.seed, L.vlen, h->st);
      } else {
        if (!tv_random[l]) fail(DDAMG_ERR_ARG, "random test vectors of a coarse level missing");
        import_fields(h, L, L.tv64 + (size_t)take * L.vlen, tv_random[l], L.N - take);
      }
    }
  }
  sync(h);
  if (h->p.precision != 0) setup_smooth<float>(h, l);
  else setup_smooth<double>(h, l);
  rebuild(h, l);
  if (l < h->L - 2) initial_setup_phase(h, l + 1, tv_random);
}

// Alg. 4 on level l: every test vector of the level goes through one K-cycle; the results (and the
// last iterates on the coarser levels) replace the test vectors, normalised.  Within one pass P and
// the coarse operators do not change, so the K-cycles of different test vectors are independent:
// they run in batches of up to work_batch columns, with results identical bit for bit to one
// vector at a time (every kernel treats the columns of a batch independently).  That holds for the
// levels l and l+1, whose values are the cycle's output and the result of the one level-(l+1)
// solve.  A level l+2 or deeper takes the last iterate of a solver that the level-(l+1) FGMRES
// calls once per step, and in a batch those calls go on for a column after its own level-(l+1)
// solve has converged (with a zero direction), which overwrites its last iterate; so a pass that
// updates such levels (l <= L-4) runs one test vector at a time.
template <typename T>
void iterative_setup_phase(ddamg_handle* h, int l, int i) {
  if (l >= h->L - 1) return;
  Level& L = h->lv[l];
  cudaStream_t st = h->st;
  const int cb = l + 2 <= h->L - 2 ? 1 : std::max(1, std::min(h->work_batch, h->setup_batch));
  cplx<T>* bT = static_cast<cplx<T>*>(scratch(h, 5, sizeof(cplx<T>) * L.vlen * cb));
  cplx<T>* zT = static_cast<cplx<T>*>(scratch(h, 6, sizeof(cplx<T>) * L.vlen * cb));
  double* nrm = static_cast<double*>(scratch(h, 7, sizeof(double) * 64));
  for (int j0 = 0; j0 < L.N; j0 += cb) {
    SetupTimer tm{h, l, DDAMG_SETUP_KCYCLE};
    const int jb = std::min(cb, L.N - j0);
    blas_convert<T, double>(bT, L.tv64 + (size_t)j0 * L.vlen, L.vlen, jb, L.vlen, L.vlen, st);
    kcycle_run<T>(h, l, zT, bT, jb);
    for (int k = l; k < h->L - 1; ++k) {
      Level& K = h->lv[k];
      const int nk = std::min(jb, K.N - j0);   // columns that are test vectors of level k
      if (nk <= 0) continue;
      const cplx<T>* src = (k == l) ? zT : work<T>(K).xs;
      cplx<double>* dst = K.tv64 + (size_t)j0 * K.vlen;
      blas_convert<double, T>(dst, src, K.vlen, nk, K.vlen, K.vlen, st);
      blas_norm2<double>(nrm, dst, K.vlen, nk, K.vlen, st);
      blas_recip(nrm, nk, st);
      blas_scale_to<double>(dst, dst, nrm, K.vlen, nk, K.vlen, st);
    }
    sync(h);
  }
  for (int k = l; k < h->L - 1; ++k) rebuild(h, k);
  for (int q = 1; q <= i; ++q) iterative_setup_phase<T>(h, l + 1, q);
}

void build_hierarchy(ddamg_handle* h) {
  const ddamg_params& p = h->p;
  h->L = p.levels;
  h->lv.resize(h->L);
  int dims[4] = {h->dims[0], h->dims[1], h->dims[2], h->dims[3]};
  for (int l = 0; l < h->L; ++l) {
    Level& L = h->lv[l];
    L.idx = l;
    L.fine = l == 0;
    L.coarsest = l == h->L - 1;
    L.n = l == 0 ? 12 : 2 * h->lv[l - 1].N;
    L.N = L.coarsest ? 0 : p.n_tv[l];
    if (!L.coarsest && (L.N <= 0 || 2 * L.N > 64)) fail(DDAMG_ERR_ARG, "n_tv must be in 1..32");
    if (L.coarsest) {
      const int one[4] = {1, 1, 1, 1};
      make_geom(L.g, dims, dims, one);
      // odd-even GMRES needs even extents; otherwise plain GMRES on D_L
      L.eo = true;
      for (int d = 0; d < 4; ++d) L.eo = L.eo && dims[d] % 2 == 0;
    } else {
      // red-black SAP needs an even block count per direction (or one block): a
      // block that gives an odd count is widened to the smallest extent that
      // divides the lattice into an even count
      int B[4];
      for (int d = 0; d < 4; ++d) {
        int c = p.sap_block[l][d];
        while (c < dims[d] && (dims[d] % c != 0 || (dims[d] / c) % 2 != 0)) ++c;
        B[d] = c < dims[d] ? c : dims[d];
      }
      make_geom(L.g, dims, p.agg[l], B, l > 0);
    }
    L.vlen = (size_t)L.g.V * L.n;
    if (!L.coarsest)
      for (int d = 0; d < 4; ++d) dims[d] /= p.agg[l][d];
  }
}

// workspaces of one precision on every level: inner FGMRES on levels 1..L-2,
// GMRES on the coarsest, K-cycle input/output on level 0
template <typename T>
void ensure_work(ddamg_handle* h) {
  bool& ready = h->work_ready[sizeof(T) == 4 ? 1 : 0];
  if (ready) return;
  if (h->cap.active) fail(DDAMG_ERR_ARG, "workspace allocation inside a graph capture");
  for (int l = 0; l < h->L; ++l) {
    Level& L = h->lv[l];
    const int m = L.coarsest ? h->p.coarse_restart : (l >= 1 ? h->p.kcycle_len : 0);
    const WorkRole role = L.fine ? WORK_FINE : (L.coarsest ? WORK_COARSEST : WORK_COARSE);
    alloc_work<T>(h, L, work<T>(L), m, role, h->work_batch);
  }
  ready = true;
}

// reduction scratch of a stream this handle launches on, sized for its largest reductions
// (reserved before any capture, so that captured graphs never see it grow)
void reserve_stream_partials(ddamg_handle* h, cudaStream_t st) {
  int mx = h->p.outer_restart;
  if (h->p.coarse_restart > mx) mx = h->p.coarse_restart;
  int bmax = h->max_batch > h->work_batch ? h->max_batch : h->work_batch;
  for (auto& L : h->lv)
    if (L.N > bmax) bmax = L.N;
  reserve_partials(bmax, mx + 1, st);
}

void allocate_hierarchy(ddamg_handle* h) {
  kry_prepare();
  const int B = h->max_batch;
  for (int l = 0; l < h->L; ++l) {
    Level& L = h->lv[l];
    if (L.fine) {
      L.f64.g = L.f32.g = L.g;
      L.f64.bc_t = L.f32.bc_t = h->bc_t;
      L.f64.U = dalloc<cplx<double>>(h, (size_t)36 * L.g.V);
      L.f32.U = dalloc<cplx<float>>(h, (size_t)36 * L.g.V);
      L.f64.clov = dalloc<double>(h, (size_t)72 * L.g.V);
      L.f32.clov = dalloc<float>(h, (size_t)72 * L.g.V);
    } else {
      L.c64.g = L.c32.g = L.g;
      L.c64.n = L.c32.n = L.n;
      const size_t nb = (size_t)L.g.V * 9 * L.n * L.n;
      L.c64.blk = dalloc<cplx<double>>(h, nb);
      L.c32.blk = dalloc<cplx<float>>(h, nb);
      if (L.coarsest && L.eo) {
        L.c64.selfinv = dalloc<cplx<double>>(h, (size_t)L.g.V * L.n * L.n);
        L.c32.selfinv = dalloc<cplx<float>>(h, (size_t)L.g.V * L.n * L.n);
        std::vector<int> odd;
        for (int x = 0; x < L.g.V; ++x) {
          int c[4];
          geom_coords(L.g, x, c);
          if (geom_parity(c) == 1) odd.push_back(x);
        }
        int* d = dalloc<int>(h, odd.size());
        CK(cudaMemcpy(d, odd.data(), sizeof(int) * odd.size(), cudaMemcpyHostToDevice));
        L.c64.odd_sites = L.c32.odd_sites = d;
        L.c64.n_odd = L.c32.n_odd = (int)odd.size();
        // tables of the cluster solver: even/odd lists and the list index of each neighbour
        std::vector<int> even, pos(L.g.V, -1);
        for (int x = 0; x < L.g.V; ++x) {
          int c[4];
          geom_coords(L.g, x, c);
          if (geom_parity(c) == 0) even.push_back(x);
        }
        for (size_t q = 0; q < even.size(); ++q) pos[even[q]] = (int)q;
        for (size_t q = 0; q < odd.size(); ++q) pos[odd[q]] = (int)q;
        auto nbr_table = [&](const std::vector<int>& from) {
          std::vector<int> t(from.size() * 8);
          for (size_t q = 0; q < from.size(); ++q) {
            int c[4];
            geom_coords(L.g, from[q], c);
            for (int k = 0; k < 8; ++k) t[q * 8 + k] = pos[geom_neighbor(L.g, c, k % 4, k < 4 ? +1 : -1)];
          }
          return t;
        };
        const std::vector<int> eo = nbr_table(odd), oe = nbr_table(even);
        int* de = dalloc<int>(h, even.size());
        int* deo = dalloc<int>(h, eo.size());
        int* doe = dalloc<int>(h, oe.size());
        CK(cudaMemcpy(de, even.data(), sizeof(int) * even.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(deo, eo.data(), sizeof(int) * eo.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(doe, oe.data(), sizeof(int) * oe.size(), cudaMemcpyHostToDevice));
        h->cgeo.even = de;
        h->cgeo.odd = d;
        h->cgeo.nbr_e_of_o = deo;
        h->cgeo.nbr_o_of_e = doe;
        h->cgeo.n_even = (int)even.size();
        h->cgeo.n_odd = (int)odd.size();
        CoarsestPlanIn in{(int)even.size(), (int)odd.size(), L.n, h->p.coarse_restart};
        h->have_cplan32 = coarsest_cluster_plan<float>(in, &h->cplan32) != 0;
        h->have_cplan64 = coarsest_cluster_plan<double>(in, &h->cplan64) != 0;
        cudaGetLastError();
      }
    }
    if (!L.fine && !L.coarsest) {
      int cls = 0, spc = 0;
      L.c32.sap_cls = coarse_sap_cluster_plan<float>(L.g, L.n, &cls, &spc, &L.c32.sap_nsl) ? cls : 0;
      L.c64.sap_cls = coarse_sap_cluster_plan<double>(L.g, L.n, &cls, &spc, &L.c64.sap_nsl) ? cls : 0;
      cudaGetLastError();
    }
    if (!L.coarsest) {
      L.tv64 = dalloc<cplx<double>>(h, L.vlen * L.N);
      L.P64 = dalloc<cplx<double>>(h, L.vlen * L.N);
      L.P32 = dalloc<cplx<float>>(h, L.vlen * L.N);
      build_block_lists(h, L);
    }
  }
  // workspaces of the configured preconditioner precision (the other precision's are
  // allocated by the first per-operation call that uses them)
  if (h->p.precision != 0) ensure_work<float>(h);
  else ensure_work<double>(h);
  alloc_work<double>(h, h->lv[0], h->outer, h->p.outer_restart, WORK_OUTER, B);
  h->ob = dalloc<cplx<double>>(h, h->lv[0].vlen * B);
  h->ox = dalloc<cplx<double>>(h, h->lv[0].vlen * B);
  h->pin32 = dalloc<cplx<float>>(h, h->lv[0].vlen * B);
  h->pout32 = dalloc<cplx<float>>(h, h->lv[0].vlen * B);
  reserve_stream_partials(h, h->st);
  for (int d = 0; d < 12; ++d)
    if (h->cap.s[d]) reserve_stream_partials(h, h->cap.s[d]);
}

void validate(const ddamg_params& p) {
  if (p.levels < 2 || p.levels > DDAMG_MAX_LEVELS) fail(DDAMG_ERR_ARG, "levels must be 2..4");
  if (p.outer_restart < 1 || p.outer_restart > 63 || p.coarse_restart < 1 || p.coarse_restart > 63 ||
      p.kcycle_len < 1 || p.kcycle_len > 63)
    fail(DDAMG_ERR_ARG, "Krylov lengths must be 1..63");
  if (p.mr_steps < 0 || p.nu < 0 || p.mu < 0 || p.n_inv < 0 || p.eta_passes < 0) fail(DDAMG_ERR_ARG, "negative count");
  if (p.max_rhs < 1 || p.max_rhs > 64) fail(DDAMG_ERR_ARG, "max_rhs must be 1..64");
  if (p.setup_batch < 0 || p.setup_batch > 64) fail(DDAMG_ERR_ARG, "setup_batch must be 0..64");
  if (p.precision < 0 || p.precision > 2) fail(DDAMG_ERR_ARG, "precision must be 0, 1 or 2");
}

template <typename T>
void precond_outer(ddamg_handle* h, cplx<double>* z, const cplx<double>* v, int nrhs);

template <>
void precond_outer<double>(ddamg_handle* h, cplx<double>* z, const cplx<double>* v, int nrhs) {
  Prof pr(h, DDAMG_PROF_PRECOND, 0.0);
  kcycle_run<double>(h, 0, z, v, nrhs);
}

template <>
void precond_outer<float>(ddamg_handle* h, cplx<double>* z, const cplx<double>* v, int nrhs) {
  const size_t vl = h->lv[0].vlen;
  Prof pr(h, DDAMG_PROF_PRECOND, 0.0);
  blas_convert<float, double>(h->pin32, v, vl, nrhs, vl, vl, h->st);
  kcycle_run<float>(h, 0, h->pout32, h->pin32, nrhs);
  blas_convert<double, float>(z, h->pout32, vl, nrhs, vl, vl, h->st);
}

// ---------------------------------------------------------------------------
// The plain Krylov solver the paper compares with (Sec. 3.3): CGNR, here in its least-squares
// form (CG on D^+ D x = D^+ b that updates s = b - D x), in FP64 on the fine operator, with
// D^+ = Gamma_5 D Gamma_5 (gamma_5-symmetry, Sec. 1).  Batched over right-hand sides, each with
// its own coefficients; a column stops when ||s|| <= tol ||b|| and its true residual is
// recomputed at the end.
void cg_alloc(ddamg_handle* h) {
  if (h->cg_vec) return;
  h->cg_vec = dalloc<cplx<double>>(h, (size_t)4 * h->max_batch * h->lv[0].vlen);
  h->cg_coef = dalloc<cplx<double>>(h, 64);
  h->cg_dcoef = dalloc<double>(h, 64);
  CK(cudaMallocHost(&h->cg_host, sizeof(double) * 4 * 64));
}

void cg_norms(ddamg_handle* h, const cplx<double>* v, int nb, double* host) {
  Level& F = h->lv[0];
  double* d = h->cg_dcoef;
  blas_norm2<double>(d, v, F.vlen, nb, F.vlen, h->st);
  CK(cudaMemcpyAsync(host, d, sizeof(double) * nb, cudaMemcpyDeviceToHost, h->st));
  sync(h);
}

void cgnr_batch(ddamg_handle* h, int nb, double tol, int max_iter, KrylovResult* res) {
  cg_alloc(h);
  Level& F = h->lv[0];
  const size_t vl = F.vlen, vs = (size_t)h->max_batch * vl;
  cplx<double>*s = h->cg_vec, *r = s + vs, *p = r + vs, *q = p + vs;
  cplx<double>* x = h->ox;
  const cplx<double>* b = h->ob;
  cudaStream_t st = h->st;
  auto D = [&](cplx<double>* o, const cplx<double>* i) { apply_D<double>(h, F, o, i, nullptr, nb); };
  auto DH = [&](cplx<double>* o, const cplx<double>* i, cplx<double>* tmp) {   // o = Gamma_5 D Gamma_5 i
    fine_gamma5(tmp, i, F.g.V, nb, vl, st);
    D(o, tmp);
    fine_gamma5(o, o, F.g.V, nb, vl, st);
  };
  double* hv = h->cg_host;   // [0, 64): per-column scalars read back; [64, 128): coefficients
  std::vector<double> bn(nb), gam(nb);
  std::vector<int> done(nb, 0), its(nb, 0);
  cg_norms(h, b, nb, hv);
  for (int c = 0; c < nb; ++c) {
    bn[c] = hv[c];
    done[c] = bn[c] == 0.0;
  }
  blas_zero<double>(x, vl, nb, vl, st);
  blas_convert<double, double>(s, b, vl, nb, vl, vl, st);
  DH(r, s, q);
  blas_convert<double, double>(p, r, vl, nb, vl, vl, st);
  cg_norms(h, r, nb, hv);
  for (int c = 0; c < nb; ++c) gam[c] = hv[c] * hv[c];
  auto upload_axpy = [&](const std::vector<double>& a) {
    for (int c = 0; c < nb; ++c) {
      hv[64 + 2 * c] = a[c];
      hv[64 + 2 * c + 1] = 0.0;
    }
    CK(cudaMemcpyAsync(h->cg_coef, hv + 64, sizeof(cplx<double>) * nb, cudaMemcpyHostToDevice, st));
  };
  std::vector<double> coef(nb);
  for (int it = 0; it < max_iter; ++it) {
    bool all = true;
    for (int c = 0; c < nb; ++c) all = all && done[c];
    if (all) break;
    D(q, p);
    cg_norms(h, q, nb, hv);
    for (int c = 0; c < nb; ++c) coef[c] = (done[c] || hv[c] == 0.0) ? 0.0 : gam[c] / (hv[c] * hv[c]);
    upload_axpy(coef);
    blas_multiaxpy<double>(x, p, 0, 1, h->cg_coef, 1, 1.0, vl, nb, vl, st);
    blas_multiaxpy<double>(s, q, 0, 1, h->cg_coef, 1, -1.0, vl, nb, vl, st);
    cg_norms(h, s, nb, hv);
    for (int c = 0; c < nb; ++c)
      if (!done[c]) {
        its[c] = it + 1;
        if (hv[c] <= tol * bn[c]) done[c] = 1;
      }
    DH(r, s, q);
    cg_norms(h, r, nb, hv);
    for (int c = 0; c < nb; ++c) {
      const double g2 = hv[c] * hv[c];
      coef[c] = (done[c] || gam[c] == 0.0) ? 0.0 : g2 / gam[c];
      gam[c] = g2;
    }
    for (int c = 0; c < nb; ++c) hv[128 + c] = coef[c];
    CK(cudaMemcpyAsync(h->cg_dcoef, hv + 128, sizeof(double) * nb, cudaMemcpyHostToDevice, st));
    blas_scale_to<double>(p, p, h->cg_dcoef, vl, nb, vl, st);
    blas_axpy<double>(p, r, 1.0, vl, nb, vl, st);
  }
  // true residuals b - D x
  apply_D<double>(h, F, s, x, b, nb);
  cg_norms(h, s, nb, hv);
  res->iterations.assign(nb, 0);
  res->cycles.assign(nb, 1);
  res->converged.assign(nb, 0);
  res->true_residual.assign(nb, 0.0);
  for (int c = 0; c < nb; ++c) {
    res->iterations[c] = its[c];
    res->true_residual[c] = bn[c] > 0 ? hv[c] / bn[c] : 0.0;
    res->converged[c] = res->true_residual[c] <= tol;
  }
}

// number of eigenvalues below x of the symmetric tridiagonal matrix (d, off-diagonal squares e2)
int sturm_count(const std::vector<double>& d, const std::vector<double>& e2, double x) {
  int cnt = 0;
  double q = d[0] - x;
  if (q < 0) ++cnt;
  for (size_t i = 1; i < d.size(); ++i) {
    if (q == 0.0) q = 1e-300;
    q = d[i] - x - e2[i - 1] / q;
    if (q < 0) ++cnt;
  }
  return cnt;
}

// the k-th smallest eigenvalue (k = 0..n-1) by bisection on the Sturm count
double tridiag_eig(const std::vector<double>& d, const std::vector<double>& e2, int k) {
  const size_t n = d.size();
  double lo = 1e300, hi = -1e300;
  for (size_t i = 0; i < n; ++i) {
    double rad = 0;
    if (i > 0) rad += std::sqrt(e2[i - 1]);
    if (i + 1 < n) rad += std::sqrt(e2[i]);
    lo = std::min(lo, d[i] - rad);
    hi = std::max(hi, d[i] + rad);
  }
  for (int it = 0; it < 300 && hi - lo > 1e-15 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count(d, e2, mid) > k) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Smallest and largest singular value of D from the Lanczos matrix of CG on D^+ D (Saad, Sec. 6.7.3:
// diagonal 1/alpha_j + beta_{j-1}/alpha_{j-1}, off-diagonal sqrt(beta_j)/alpha_j), started from a
// seeded random field; the extreme Ritz values approach lambda_min and lambda_max of D^+ D.
void sigma_extremes(ddamg_handle* h, int steps, uint64_t seed, double* smin, double* smax, int* used) {
  cg_alloc(h);
  Level& F = h->lv[0];
  const size_t vl = F.vlen, vs = (size_t)h->max_batch * vl;
  cplx<double>*s = h->cg_vec, *r = s + vs, *p = r + vs, *q = p + vs;
  cudaStream_t st = h->st;
  double* hv = h->cg_host;
  draw_fields(r, F.g, true, F.n, 1, 0, 7, seed, vl, st);
  blas_convert<double, double>(p, r, vl, 1, vl, vl, st);
  cg_norms(h, r, 1, hv);
  double gam = hv[0] * hv[0];
  const double gam0 = gam;
  std::vector<double> al, be;
  for (int j = 0; j < steps; ++j) {
    apply_D<double>(h, F, q, p, nullptr, 1);      // q = D p, <p, D^+ D p> = |q|^2
    cg_norms(h, q, 1, hv);
    if (!(hv[0] > 0.0)) break;
    const double alpha = gam / (hv[0] * hv[0]);
    fine_gamma5(s, q, F.g.V, 1, vl, st);           // s = D^+ q = Gamma_5 D Gamma_5 q
    apply_D<double>(h, F, q, s, nullptr, 1);
    fine_gamma5(s, q, F.g.V, 1, vl, st);
    hv[64] = -alpha;
    hv[65] = 0.0;
    CK(cudaMemcpyAsync(h->cg_coef, hv + 64, sizeof(cplx<double>), cudaMemcpyHostToDevice, st));
    blas_multiaxpy<double>(r, s, 0, 1, h->cg_coef, 1, 1.0, vl, 1, vl, st);   // r -= alpha D^+ D p
    cg_norms(h, r, 1, hv);
    const double g2 = hv[0] * hv[0];
    al.push_back(alpha);
    be.push_back(g2 / gam);
    if (g2 <= 1e-28 * gam0) break;
    hv[128] = g2 / gam;
    CK(cudaMemcpyAsync(h->cg_dcoef, hv + 128, sizeof(double), cudaMemcpyHostToDevice, st));
    blas_scale_to<double>(p, p, h->cg_dcoef, vl, 1, vl, st);
    blas_axpy<double>(p, r, 1.0, vl, 1, vl, st);
    gam = g2;
  }
  const size_t k = al.size();
  if (k == 0) fail(DDAMG_ERR_ARG, "no Lanczos step could be taken");
  std::vector<double> d(k), e2(k > 1 ? k - 1 : 1, 0.0);
  for (size_t j = 0; j < k; ++j) {
    d[j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
    if (j + 1 < k) e2[j] = be[j] / (al[j] * al[j]);
  }
  *smin = std::sqrt(std::max(0.0, tridiag_eig(d, e2, 0)));
  *smax = std::sqrt(std::max(0.0, tridiag_eig(d, e2, (int)k - 1)));
  if (used) *used = (int)k;
}

}  // namespace

namespace {
int guard(const std::function<void()>& f) {
  try {
    f();
    return DDAMG_OK;
  } catch (const DdError& e) {
    g_err = e.msg;
    return e.code;
  } catch (const std::exception& e) {
    g_err = e.what();
    return DDAMG_ERR_ARG;
  }
}

Level& level_of(ddamg_handle* h, int level) {
  if (!h || level < 0 || level >= h->L) fail(DDAMG_ERR_ARG, "level out of range");
  return h->lv[level];
}

// run f on n fields of level l in chunks of the batch size; in/out are ABI (FP64 lex) buffers
template <typename T, class F>
void hook(ddamg_handle* h, int l, const double* in, double* out, int n, bool out_is_in_out, int out_level, F f) {
  ensure_work<T>(h);
  Level& L = h->lv[l];
  Level& O = h->lv[out_level];
  const size_t in_bytes = sizeof(cplx<double>) * L.vlen * n;
  const size_t out_bytes = sizeof(cplx<double>) * O.vlen * n;
  const cplx<double>* din = in ? static_cast<const cplx<double>*>(dev_in(h, in, in_bytes, 0)) : nullptr;
  const bool out_dev = is_device_ptr(out);
  cplx<double>* dout = out_dev ? reinterpret_cast<cplx<double>*>(out)
                               : static_cast<cplx<double>*>(scratch(h, 1, out_bytes));
  if (!out_dev && out_is_in_out) CK(cudaMemcpyAsync(dout, out, out_bytes, cudaMemcpyHostToDevice, h->st));
  cplx<T>* ti = static_cast<cplx<T>*>(scratch(h, 2, sizeof(cplx<T>) * L.vlen * n));
  cplx<T>* to = static_cast<cplx<T>*>(scratch(h, 3, sizeof(cplx<T>) * O.vlen * n));
  auto imp = [&](Level& X, cplx<T>* dst, const cplx<double>* src) {
    if (X.fine) fine_import<T>(dst, src, X.g, n, X.vlen, h->st);
    else coarse_import<T>(dst, src, X.g, X.n, n, X.vlen, h->st);
  };
  auto exp = [&](Level& X, cplx<double>* dst, const cplx<T>* src) {
    if (X.fine) fine_export<T>(dst, src, X.g, n, X.vlen, h->st);
    else coarse_export<T>(dst, src, X.g, X.n, n, X.vlen, h->st);
  };
  if (din) imp(L, ti, din);
  if (out_is_in_out) imp(O, to, dout);
  f(to, ti);
  exp(O, dout, to);
  if (!out_dev) CK(cudaMemcpyAsync(out, dout, out_bytes, cudaMemcpyDeviceToHost, h->st));
  sync(h);
}

}  // namespace

// ===========================================================================
// C ABI
namespace {

// The outer FGMRES (FP64, flexible, preconditioned by one K-cycle) on the first
// nb right-hand sides of h->ob, iterate in h->ox.  resume: continue from h->ox
// and its residual in h->outer.r (one restart cycle at a time, as the serving
// loop runs it).
void outer_fgmres(ddamg_handle* h, int nb, double tol, int max_cycles, KrylovResult* res, bool resume = false,
                  const double* tol_rhs = nullptr) {
  Level& F = h->lv[0];
  const bool df = h->outer_df && F.Udf;
  auto A = [&](cplx<double>* o, const cplx<double>* in, const cplx<double>* bb) {
    if (df && !bb) {   // D z_j of the Arnoldi step; residuals b - D x stay FP64
      Prof pr(h, DDAMG_PROF_FINE_DSLASH, (double)F.vlen * 16 * nb * 2 + (double)F.g.V * (36 * 16 + 72 * 8));
      fine_dslash_df(o, in, nullptr, F.Udf, F.clovdf, F.g, F.f64.bc_t, nb, F.vlen, h->st);
    } else {
      apply_D<double>(h, F, o, in, bb, nb);
    }
  };
  auto M = [&](cplx<double>* z, const cplx<double>* v) {
    if (h->p.precision != 0) precond_outer<float>(h, z, v, nb);
    else precond_outer<double>(h, z, v, nb);
  };
  krylov_host<double>(h, h->outer, F.vlen, h->ox, h->ob, nb, h->p.outer_restart, tol, max_cycles, true, true, A, M,
                      res, resume, tol_rhs, df);
}

// ---------------------------------------------------------------------------
// Serving: continuous batching of right-hand sides over resident hierarchies.
//
// Each registered hierarchy has a worker thread and keeps using the handle's
// own stream, so the work of different hierarchies overlaps on the device.
// Requests (1..n right-hand sides, one tolerance) are split into columns that
// wait in a FIFO queue; a column enters a free batch slot at the next restart
// boundary of the outer FGMRES, the batch runs one restart cycle, and slots
// whose true residual meets their tolerance (or that used up the restart
// budget) leave it; the remaining slots are compacted to the front.  Every
// right-hand side is computed with batch-independent reductions, so its
// iterate is the same whichever other columns share its batch.

double now_seconds() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct SrvRequest {
  int hid = 0, n = 0;
  double tol = 0;
  std::vector<double> b, x;   // n fields in the ABI layout
  std::vector<ddamg_stats> st;
  int remaining = 0;
  int status = 1;             // 1: pending; 0: done; < 0: DDAMG_ERR_* of the request
  std::string err;            // the worker's error message of a failed request
  double t_submit = 0, t_start = 0, t_done = 0;
};

struct SrvSlot {
  SrvRequest* rq = nullptr;
  int col = 0, iterations = 0, cycles = 0;
};

struct SrvHier {
  ddamg_handle* h = nullptr;
  std::deque<std::pair<SrvRequest*, int>> queue;   // columns waiting for a slot
  std::vector<SrvSlot> slots;                      // slots [0, active) are in the batch
  int active = 0;
  size_t bytes = 0;
  std::thread worker;
};

}  // namespace

struct ddamg_server {
  std::mutex mu;
  std::condition_variable work_cv, done_cv;
  std::vector<SrvHier*> hs;
  std::map<long long, SrvRequest*> reqs;
  long long next_id = 1;
  bool stop = false;
  size_t budget = 0, used = 0;
};

namespace {

void finish_column(ddamg_server* S, SrvRequest* rq, int col, const ddamg_stats& st, int err,
                   const std::string& msg = std::string()) {
  rq->st[col] = st;
  if (err) {
    rq->status = err;
    if (rq->err.empty()) rq->err = msg;
  }
  if (--rq->remaining == 0) {
    if (rq->status == 1) {
      bool ok = true;
      for (const auto& q : rq->st) ok = ok && q.converged;
      rq->status = ok ? DDAMG_OK : DDAMG_ERR_NOCONV;
    }
    rq->t_done = now_seconds();
    S->done_cv.notify_all();
  }
}

void server_worker(ddamg_server* S, SrvHier* H) {
  ddamg_handle* h = H->h;
  cudaSetDevice(h->device);
  Level& F = h->lv[0];
  const size_t vlen = F.vlen;
  const size_t fb = sizeof(cplx<double>) * vlen;
  const int cap = h->max_batch;
  H->slots.assign(cap, SrvSlot{});
  std::vector<double> tols(cap);
  for (;;) {
    std::vector<int> fresh;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->work_cv.wait(lk, [&] { return S->stop || !H->queue.empty() || H->active > 0; });
      if (S->stop && H->active == 0) {
        for (auto& qc : H->queue) finish_column(S, qc.first, qc.second, ddamg_stats{}, DDAMG_ERR_ARG);
        H->queue.clear();
        return;
      }
      while (!S->stop && H->active < cap && !H->queue.empty()) {
        SrvSlot sl;
        sl.rq = H->queue.front().first;
        sl.col = H->queue.front().second;
        H->queue.pop_front();
        if (sl.rq->t_start == 0) sl.rq->t_start = now_seconds();
        H->slots[H->active] = sl;
        fresh.push_back(H->active++);
      }
    }
    const int na = H->active;
    std::vector<int> retire;
    std::vector<ddamg_stats> rst;
    const int rc = guard([&] {
      for (int q : fresh) {   // new columns: b into the slot, x = 0, r = b
        const SrvSlot& sl = H->slots[q];
        const cplx<double>* din =
            static_cast<const cplx<double>*>(dev_in(h, sl.rq->b.data() + (size_t)sl.col * vlen * 2, fb, 0));
        fine_import<double>(h->ob + (size_t)q * vlen, din, F.g, 1, vlen, h->st);
        blas_zero<double>(h->ox + (size_t)q * vlen, vlen, 1, vlen, h->st);
        CK(cudaMemcpyAsync(h->outer.r + (size_t)q * vlen, h->ob + (size_t)q * vlen, fb, cudaMemcpyDeviceToDevice,
                           h->st));
      }
      for (int q = 0; q < na; ++q) tols[q] = H->slots[q].rq->tol;
      KrylovResult res;
      outer_fgmres(h, na, 1.0, 1, &res, true, tols.data());
      int e = 0;
      CK(cudaMemcpyAsync(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
      sync(h);
      if (e == 2) {
        CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->st));
        fail(DDAMG_ERR_CUDA, "a shared-memory staging wait of the SAP kernel timed out");
      }
      cplx<double>* dx = static_cast<cplx<double>*>(scratch(h, 1, fb));
      for (int q = 0; q < na; ++q) {
        SrvSlot& sl = H->slots[q];
        sl.iterations += res.iterations[q];
        sl.cycles += 1;
        if (!(res.converged[q] || sl.cycles >= h->p.outer_max_cycles)) continue;
        ddamg_stats st;
        st.iterations = sl.iterations;
        st.cycles = sl.cycles;
        st.converged = res.converged[q];
        st.true_residual = res.true_residual[q];
        fine_export<double>(dx, h->ox + (size_t)q * vlen, F.g, 1, vlen, h->st);
        CK(cudaMemcpyAsync(sl.rq->x.data() + (size_t)sl.col * vlen * 2, dx, fb, cudaMemcpyDeviceToHost, h->st));
        sync(h);
        retire.push_back(q);
        rst.push_back(st);
      }
      // compact: the last slots move into the holes (b, x and the residual of the iterate)
      int act = na;
      for (int k = (int)retire.size() - 1; k >= 0; --k) {
        const int q = retire[k], last = act - 1;
        if (q != last) {
          for (cplx<double>* base : {h->ob, h->ox, h->outer.r})
            CK(cudaMemcpyAsync(base + (size_t)q * vlen, base + (size_t)last * vlen, fb, cudaMemcpyDeviceToDevice,
                               h->st));
        }
        --act;
      }
      sync(h);
    });
    std::lock_guard<std::mutex> lk(S->mu);
    if (rc != DDAMG_OK) {   // the batch failed: every column in it fails, with the worker's message
      for (int q = 0; q < na; ++q) finish_column(S, H->slots[q].rq, H->slots[q].col, ddamg_stats{}, rc, g_err);
      H->active = 0;
      continue;
    }
    for (size_t k = 0; k < retire.size(); ++k) {
      const SrvSlot& sl = H->slots[retire[k]];
      finish_column(S, sl.rq, sl.col, rst[k], 0);
    }
    int act = na;
    for (int k = (int)retire.size() - 1; k >= 0; --k) {
      const int q = retire[k], last = act - 1;
      if (q != last) H->slots[q] = H->slots[last];
      --act;
    }
    H->active = act;
  }
}

// Device bytes of a hierarchy with these parameters, before it is built: the
// allocations of the setup (operators, P, test vectors, Krylov workspaces, FP16
// copies) and the staging buffers of a full batch.
size_t estimate_bytes(const int dims0[4], const ddamg_params& p) {
  size_t tot = 0;
  const size_t B = (size_t)p.max_rhs;
  // level workspaces hold max(max_rhs, setup batch) columns (Alg. 4 runs in batches)
  const size_t WB = std::max(B, (size_t)std::min(p.setup_batch > 0 ? p.setup_batch : 4, 64));
  int dims[4] = {dims0[0], dims0[1], dims0[2], dims0[3]};
  int nprev = 12, Nprev = 0;
  size_t vlen0 = 0, maxtmp = 0;
  for (int l = 0; l < p.levels; ++l) {
    const bool fine = l == 0, coarsest = l == p.levels - 1;
    const size_t V = (size_t)dims[0] * dims[1] * dims[2] * dims[3];
    const int n = fine ? 12 : 2 * Nprev;
    const size_t vlen = V * n;
    const int N = coarsest ? 0 : p.n_tv[l];
    if (fine) {
      vlen0 = vlen;
      tot += 36 * V * (16 + 8) + 72 * V * (8 + 4);
      if (p.precision == 2) tot += 36 * V * 4 + 72 * V * 2;
    } else {
      const size_t nb = V * 9 * (size_t)n * n;
      tot += nb * (16 + 8) + (p.precision == 2 ? nb * 4 + V * 4 : 0);
      if (coarsest) tot += V * (size_t)n * n * (16 + 8) + 4 * V * sizeof(int) + 16 * V * sizeof(int);
    }
    if (!coarsest) {
      tot += vlen * N * (16 + 16 + 8) + (p.precision == 2 ? vlen * N * 4 + V * 8 : 0);
      tot += (size_t)(V + 1) * sizeof(int);   // SAP block lists
      maxtmp = std::max(maxtmp, vlen * (size_t)std::min(N, 4) * 16);
    }
    // workspaces of the configured precision (see alloc_work / ensure_work)
    const int m = coarsest ? p.coarse_restart : (l >= 1 ? p.kcycle_len : 0);
    const size_t vl = vlen * WB;
    const size_t tb = p.precision == 0 ? 16 : 8;
    size_t nvec = fine ? 3 : (coarsest ? 12 : 7);
    if (m > 0) nvec += (size_t)(m + 1) + (coarsest ? 0 : (size_t)m);
    tot += nvec * vl * tb;
    const size_t mm = m > 0 ? m : 1;
    tot += WB * ((mm + 1) * mm * 16 + mm * 8 + mm * 16 + 4 * (mm + 1) * 16 + 64);
    if (!coarsest) {
      for (int d = 0; d < 4; ++d) dims[d] /= p.agg[l][d];
      nprev = n;
      Nprev = N;
    }
  }
  (void)nprev;
  const size_t vl0 = vlen0 * B;
  tot += (size_t)(2 * p.outer_restart + 2) * vl0 * 16;        // outer FGMRES V, Z and residual
  tot += vl0 * (16 + 16 + 8 + 8);                              // ob, ox, pin32, pout32
  // staging: slot 0 holds the largest of the gauge field, a chunk of test vectors and a batch
  // of right-hand sides; a second slot a batch of solutions; then the setup scratch
  const size_t V0 = vlen0 / 12;
  tot += std::max({V0 * 576, vlen0 * (size_t)std::min(p.n_tv[0], 4) * 16, vl0 * 16}) + vl0 * 16;
  tot += maxtmp + 2 * maxtmp / 2;
  // Alg. 4 input and output of one batch of test vectors (setup scratch)
  tot += 2 * vlen0 * (WB > B ? WB : B) * (p.precision == 0 ? 16 : 8);
  return tot;
}

// compute precision of the per-operation entry points: 0 FP64, 1 FP32 (on the
// FP32 or FP16 storage the handle holds)
bool fp32_compute(int precision) {
  if (precision != 0 && precision != 1) fail(DDAMG_ERR_ARG, "precision must be 0 (FP64) or 1 (FP32)");
  return precision == 1;
}

}  // namespace

extern "C" {

void ddamg_default_params(ddamg_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->levels = 3;
  for (int l = 0; l < DDAMG_MAX_LEVELS; ++l)
    for (int d = 0; d < 4; ++d) {
      p->agg[l][d] = l == 0 ? 4 : 2;
      p->sap_block[l][d] = 2;
    }
  for (int l = 0; l < DDAMG_MAX_LEVELS; ++l) p->n_tv[l] = 20;
  p->mr_steps = 3;
  p->nu = 5;
  p->mu = 0;
  p->n_inv = 6;
  p->eta_passes = 3;
  p->outer_restart = 10;
  p->outer_max_cycles = 100;
  p->kcycle_len = 5;
  p->kcycle_cycles = 2;
  p->kcycle_tol = 1e-1;
  p->coarse_tol = 5e-2;
  p->coarse_restart = 50;
  p->coarse_cycles = 20;
  p->precision = 1;
  p->max_rhs = 1;
  p->seed = 0;
  p->sap_schur = 0;
  p->setup_batch = 4;
}

const char* ddamg_last_error(void) { return g_err.c_str(); }

int ddamg_setup(const double* gauge, const int dims[4], int bc_t, double m0, double csw, const ddamg_params* params,
                const double* const* tv_random, ddamg_handle** out) {
  if (!out || !gauge || !dims || !params) {
    g_err = "null argument";
    return DDAMG_ERR_ARG;
  }
  *out = nullptr;
  ddamg_handle* h = new ddamg_handle();
  const int rc = guard([&] {
    validate(*params);
    h->p = *params;
    for (int d = 0; d < 4; ++d) h->dims[d] = dims[d];
    h->bc_t = bc_t;
    h->m0 = m0;
    h->csw = csw;
    h->max_batch = params->max_rhs;
    h->setup_batch = params->setup_batch > 0 ? params->setup_batch : 4;
    h->work_batch = std::max(h->max_batch, std::min(h->setup_batch, 64));
    CK(cudaGetDevice(&h->device));
    CK(cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking));
    h->st = h->own;
    for (int d = 0; d < 12; ++d) CK(cudaStreamCreateWithFlags(&h->cap.s[d], cudaStreamNonBlocking));
    CK(cudaMallocHost(&h->h_done, sizeof(int) * 64));
    CK(cudaMallocHost(&h->h_kr, sizeof(int) * 64));
    CK(cudaMallocHost(&h->h_scal, sizeof(double) * 64));
    build_hierarchy(h);
    allocate_hierarchy(h);
    h->d_err = dalloc<int>(h, 1);
    CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->st));
    h->lv[0].f64.err = h->lv[0].f32.err = h->d_err;
    for (auto& L : h->lv) L.c64.err = L.c32.err = h->d_err;
    double gg[6 * 16 * 2];
    gamma_products(gg);
    set_gamma_products(gg);
    import_operator(h, gauge);
    if (h->p.precision == 2) {
      h->half = true;
      half_alloc(h);
      half_refresh_fine(h);
      half_bind(h);
    }
    if (h->p.sap_schur) {
      if (h->p.precision == 0) fail(DDAMG_ERR_ARG, "Schur SAP block solves are an option of the FP32 preconditioner");
      schur_check(h);
      schur_tables(h);
      h->sap_schur = true;
      schur_bind(h);
    }
    sync(h);
    initial_setup_phase(h, 0, tv_random);
    for (int i = 1; i <= h->p.n_inv; ++i) {
      if (h->p.precision != 0) iterative_setup_phase<float>(h, 0, i);
      else iterative_setup_phase<double>(h, 0, i);
    }
    // the batch kernels are chosen on the finished hierarchy (the setup ran the defaults)
    if (h->half) {
      tune_kernels(h);
      free_graphs(h);
    }
    sync(h);
  });
  if (rc != DDAMG_OK) {
    ddamg_free(h);
    return rc;
  }
  *out = h;
  return DDAMG_OK;
}

void ddamg_free(ddamg_handle* h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  free_graphs(h);
  for (int d = 0; d < 12; ++d)
    if (h->cap.s[d]) cudaStreamDestroy(h->cap.s[d]);
  for (void* p : h->allocs) cudaFree(p);
  for (auto& s : h->scr)
    if (s.p) cudaFree(s.p);
  if (h->h_done) cudaFreeHost(h->h_done);
  if (h->h_kr) cudaFreeHost(h->h_kr);
  if (h->h_scal) cudaFreeHost(h->h_scal);
  if (h->cg_host) cudaFreeHost(h->cg_host);
  for (auto& v : h->ev)
    for (cudaEvent_t e : v) cudaEventDestroy(e);
  if (h->own) cudaStreamDestroy(h->own);
  delete h;
}

int ddamg_update_gauge(ddamg_handle* h, const double* gauge, int n_inv) {
  if (!h || !gauge || n_inv < 0) {
    g_err = "invalid argument";
    return DDAMG_ERR_ARG;
  }
  return guard([&] {
    sync(h);
    import_operator(h, gauge);
    if (h->lv[0].Uh) half_refresh_fine(h);
    if (h->lv[0].mix32) schur_tables(h);
    if (h->lv[0].Udf) df_refresh(h);
    // P from the current test vectors, coarse operators of the new fine operator
    for (int l = 0; l + 1 < h->L; ++l) rebuild(h, l);
    for (int i = 1; i <= n_inv; ++i) {
      if (h->p.precision != 0) iterative_setup_phase<float>(h, 0, i);
      else iterative_setup_phase<double>(h, 0, i);
    }
    sync(h);
  });
}

int ddamg_set_stream(ddamg_handle* h, void* stream) {
  if (!h) return DDAMG_ERR_ARG;
  return guard([&] {
    sync(h);
    h->st = stream ? static_cast<cudaStream_t>(stream) : h->own;
    reserve_stream_partials(h, h->st);
  });
}

int ddamg_solve(ddamg_handle* h, const double* rhs, double* x, int n, double tol, ddamg_stats* per_rhs) {
  if (!h || !rhs || !x || n < 0 || !(tol > 0)) {
    g_err = "invalid argument";
    return DDAMG_ERR_ARG;
  }
  bool all_conv = true;
  const int rc = guard([&] {
    Level& F = h->lv[0];
    const size_t fbytes = sizeof(cplx<double>) * F.vlen;
    const bool xdev = is_device_ptr(x);
    for (int s0 = 0; s0 < n; s0 += h->max_batch) {
      const int nb = (n - s0) < h->max_batch ? (n - s0) : h->max_batch;
      const cplx<double>* din =
          static_cast<const cplx<double>*>(dev_in(h, rhs + (size_t)s0 * F.vlen * 2, fbytes * nb, 0));
      fine_import<double>(h->ob, din, F.g, nb, F.vlen, h->st);
      KrylovResult res;
      outer_fgmres(h, nb, tol, h->p.outer_max_cycles, &res);
      cplx<double>* dx = xdev ? reinterpret_cast<cplx<double>*>(x + (size_t)s0 * F.vlen * 2)
                              : static_cast<cplx<double>*>(scratch(h, 1, fbytes * nb));
      fine_export<double>(dx, h->ox, F.g, nb, F.vlen, h->st);
      {
        int e = 0;
        CK(cudaMemcpyAsync(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
        sync(h);
        if (e == 2) {
          CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->st));
          fail(DDAMG_ERR_CUDA, "a shared-memory staging wait of the SAP kernel timed out");
        }
      }
      if (!xdev) CK(cudaMemcpyAsync(x + (size_t)s0 * F.vlen * 2, dx, fbytes * nb, cudaMemcpyDeviceToHost, h->st));
      sync(h);
      for (int r = 0; r < nb; ++r) {
        if (per_rhs) {
          per_rhs[s0 + r].iterations = res.iterations[r];
          per_rhs[s0 + r].cycles = res.cycles[r];
          per_rhs[s0 + r].converged = res.converged[r];
          per_rhs[s0 + r].true_residual = res.true_residual[r];
        }
        all_conv = all_conv && res.converged[r];
      }
    }
  });
  if (rc != DDAMG_OK) return rc;
  if (!all_conv) {
    g_err = "outer FGMRES did not reach the tolerance";
    return DDAMG_ERR_NOCONV;
  }
  return DDAMG_OK;
}

int ddamg_cgnr(ddamg_handle* h, const double* rhs, double* x, int n, double tol, int max_iter, ddamg_stats* per_rhs) {
  if (!h || !rhs || !x || n < 0 || !(tol > 0) || max_iter < 1) {
    g_err = "invalid argument";
    return DDAMG_ERR_ARG;
  }
  bool all_conv = true;
  const int rc = guard([&] {
    Level& F = h->lv[0];
    const size_t fbytes = sizeof(cplx<double>) * F.vlen;
    const bool xdev = is_device_ptr(x);
    for (int s0 = 0; s0 < n; s0 += h->max_batch) {
      const int nb = (n - s0) < h->max_batch ? (n - s0) : h->max_batch;
      const cplx<double>* din =
          static_cast<const cplx<double>*>(dev_in(h, rhs + (size_t)s0 * F.vlen * 2, fbytes * nb, 0));
      fine_import<double>(h->ob, din, F.g, nb, F.vlen, h->st);
      KrylovResult res;
      cgnr_batch(h, nb, tol, max_iter, &res);
      cplx<double>* dx = xdev ? reinterpret_cast<cplx<double>*>(x + (size_t)s0 * F.vlen * 2)
                              : static_cast<cplx<double>*>(scratch(h, 1, fbytes * nb));
      fine_export<double>(dx, h->ox, F.g, nb, F.vlen, h->st);
      if (!xdev) CK(cudaMemcpyAsync(x + (size_t)s0 * F.vlen * 2, dx, fbytes * nb, cudaMemcpyDeviceToHost, h->st));
      sync(h);
      for (int r = 0; r < nb; ++r) {
        if (per_rhs) {
          per_rhs[s0 + r].iterations = res.iterations[r];
          per_rhs[s0 + r].cycles = 1;
          per_rhs[s0 + r].converged = res.converged[r];
          per_rhs[s0 + r].true_residual = res.true_residual[r];
        }
        all_conv = all_conv && res.converged[r];
      }
    }
  });
  if (rc != DDAMG_OK) return rc;
  if (!all_conv) {
    g_err = "CGNR did not reach the tolerance";
    return DDAMG_ERR_NOCONV;
  }
  return DDAMG_OK;
}

int ddamg_sigma_extremes(ddamg_handle* h, int steps, uint64_t seed, double* sigma_min, double* sigma_max,
                         int* steps_taken) {
  if (!h || steps < 1 || !sigma_min) {
    g_err = "invalid argument";
    return DDAMG_ERR_ARG;
  }
  return guard([&] {
    double smax = 0.0;
    sigma_extremes(h, steps, seed, sigma_min, &smax, steps_taken);
    if (sigma_max) *sigma_max = smax;
  });
}

int ddamg_set_option(ddamg_handle* h, int option, int value) {
  if (!h) return DDAMG_ERR_ARG;
  return guard([&] {
    sync(h);
    if (option == DDAMG_OPT_GRAPHS) {
      h->use_graphs = value != 0;
    } else if (option == DDAMG_OPT_COARSEST_CLUSTER) {
      h->use_cluster = value != 0;
      free_graphs(h);   // captured graphs embed the previous choice
    } else if (option == DDAMG_OPT_SAP_CLUSTER) {
      for (auto& L : h->lv) {
        if (L.fine || L.coarsest) continue;
        int cls = 0, spc = 0;
        L.c32.sap_cls =
            (value && coarse_sap_cluster_plan<float>(L.g, L.n, &cls, &spc, &L.c32.sap_nsl, value)) ? cls : 0;
        L.c64.sap_cls =
            (value && coarse_sap_cluster_plan<double>(L.g, L.n, &cls, &spc, &L.c64.sap_nsl, value)) ? cls : 0;
      }
      cudaGetLastError();
      if (h->half) {   // the persistent SAP launch follows the cluster plan
        ensure_work<float>(h);
        tune_kernels(h);
      }
      free_graphs(h);
    } else if (option == DDAMG_OPT_HALF_STORAGE) {
      if (value && !h->lv[0].Uh) {
        half_alloc(h);
        half_refresh_fine(h);
        for (int l = 0; l + 1 < h->L; ++l) half_refresh(h, l);
        sync(h);
      }
      h->half = value != 0;
      half_bind(h);
      schur_bind(h);
      ensure_work<float>(h);
      tune_kernels(h);
      free_graphs(h);
    } else if (option == DDAMG_OPT_SAP_SCHUR) {
      if (value) {
        schur_check(h);
        if (!h->lv[0].mix32) schur_tables(h);
      }
      h->sap_schur = value != 0;
      schur_bind(h);
      free_graphs(h);
    } else if (option == DDAMG_OPT_COARSE_TC) {
      if (value < -1 || value > 4) fail(DDAMG_ERR_ARG, "coarse tensor-core option must be -1..4");
      h->tc_force = value;
      ensure_work<float>(h);
      tune_kernels(h);
      free_graphs(h);
    } else if (option == DDAMG_OPT_OUTER_DF) {
      if (value && !h->lv[0].Udf) df_refresh(h);
      h->outer_df = value != 0;
      sync(h);
    } else if (option == DDAMG_OPT_SAP_PERSIST) {
      if (value < -1 || value > 2) fail(DDAMG_ERR_ARG, "persistent SAP option must be -1, 0, 1 or 2");
      h->persist_force = value;
      ensure_work<float>(h);
      tune_kernels(h);
      free_graphs(h);
    } else {
      fail(DDAMG_ERR_ARG, "unknown option");
    }
  });
}

int ddamg_get_option(ddamg_handle* h, int option, int* value) {
  if (!h || !value) return DDAMG_ERR_ARG;
  return guard([&] {
    if (option == DDAMG_OPT_GRAPHS) {
      *value = h->use_graphs ? 1 : 0;
    } else if (option == DDAMG_OPT_COARSEST_CLUSTER) {
      *value = (h->use_cluster && h->have_cplan32) ? h->cplan32.CL : 0;
    } else if (option == DDAMG_OPT_SAP_CLUSTER) {
      *value = h->L > 2 ? h->lv[1].c32.sap_cls : 0;
    } else if (option == DDAMG_OPT_HALF_STORAGE) {
      *value = h->half ? 1 : 0;
    } else if (option == DDAMG_OPT_COARSE_TC) {
      *value = h->L > 1 ? h->lv[1].c32.tc_ks : 0;
    } else if (option == DDAMG_OPT_SAP_SCHUR) {
      *value = h->sap_schur ? 1 : 0;
    } else if (option == DDAMG_OPT_SAP_PERSIST) {
      *value = h->L > 2 ? h->lv[1].sap_persist : 0;
    } else if (option == DDAMG_OPT_OUTER_DF) {
      *value = h->outer_df ? 1 : 0;
    } else {
      fail(DDAMG_ERR_ARG, "unknown option");
    }
  });
}

int ddamg_profile(ddamg_handle* h, int enable) {
  if (!h) return DDAMG_ERR_ARG;
  return guard([&] {
    sync(h);
    if (enable) {
      for (int k = 0; k < DDAMG_PROF_KINDS; ++k) {
        h->ev_used[k] = 0;
        h->prof_bytes[k] = 0;
        h->prof_count[k] = 0;
        h->prof_graph_ms[k] = 0;
      }
    }
    h->prof = enable;
  });
}

int ddamg_profile_read(ddamg_handle* h, int kind, double* total_ms, long long* launches, double* algo_bytes) {
  if (!h || kind < 0 || kind >= DDAMG_PROF_KINDS) return DDAMG_ERR_ARG;
  return guard([&] {
    sync(h);
    double ms = h->prof_graph_ms[kind];
    for (size_t i = 0; i + 1 < h->ev_used[kind]; i += 2) {
      float t = 0;
      CK(cudaEventElapsedTime(&t, h->ev[kind][i], h->ev[kind][i + 1]));
      ms += t;
    }
    if (total_ms) *total_ms = ms;
    if (launches) *launches = h->prof_count[kind];
    if (algo_bytes) *algo_bytes = h->prof_bytes[kind];
  });
}

long long ddamg_launch_count(void) { return launch_count(); }

int ddamg_krylov_steps(ddamg_handle* h, int level, int precision, long long* steps) {
  return guard([&] {
    Level& L = level_of(h, level);
    if (!steps) fail(DDAMG_ERR_ARG, "null output");
    int dev = 0;
    long long host = 0;
    if (precision != 0) {
      if (L.w32.gs.ctl) CK(cudaMemcpy(&dev, L.w32.gs.ctl + 3, sizeof(int), cudaMemcpyDeviceToHost));
      host = L.w32.host_steps;
    } else {
      if (L.w64.gs.ctl) CK(cudaMemcpy(&dev, L.w64.gs.ctl + 3, sizeof(int), cudaMemcpyDeviceToHost));
      host = L.w64.host_steps;
    }
    *steps = host + dev + (level == 0 ? h->outer.host_steps : 0);
  });
}

int ddamg_residual_norm_noalloc(ddamg_handle* h, const double* rhs, const double* x, int n, double* out) {
  if (!h || !rhs || !x || !out) {
    g_err = "null argument";
    return DDAMG_ERR_ARG;
  }
  if (!is_device_ptr(rhs) || !is_device_ptr(x)) {
    g_err = "rhs and x must be device memory (nothing is staged: this entry point allocates nothing)";
    return DDAMG_ERR_ARG;
  }
  const char* msg = "";
  const int rc = fine_residual_norm_noalloc(out, is_device_ptr(out), reinterpret_cast<const cplx<double>*>(rhs),
                                            reinterpret_cast<const cplx<double>*>(x), h->lv[0].f64, h->device, n, h->st,
                                            &msg);
  if (rc != 0) {
    g_err = msg;
    return rc == -1 ? DDAMG_ERR_ARG : DDAMG_ERR_CUDA;
  }
  return DDAMG_OK;
}

int ddamg_autotune_times(ddamg_handle* h, int kind, int level, double* ms, int* chosen) {
  return guard([&] {
    Level& L = level_of(h, level);
    if (kind < 0 || kind > 3) fail(DDAMG_ERR_ARG, "unknown autotuned kernel");
    if (kind == DDAMG_TUNE_SAP && (L.fine || L.coarsest)) fail(DDAMG_ERR_ARG, "the coarse SAP runs on levels 1..L-2");
    if (kind == DDAMG_TUNE_COARSE && L.fine) fail(DDAMG_ERR_ARG, "the coarse stencil runs on levels >= 1");
    if (kind != DDAMG_TUNE_COARSE && L.coarsest) fail(DDAMG_ERR_ARG, "no transfer below the coarsest level");
    if (ms)
      for (int k = 0; k < 5; ++k) ms[k] = h->tune_ms[kind][level][k];
    if (chosen)
      *chosen = kind == DDAMG_TUNE_COARSE     ? L.c32.tc_ks
                : kind == DDAMG_TUNE_RESTRICT ? L.tr_ks
                : kind == DDAMG_TUNE_PROLONG  ? L.pr_batch
                                              : L.sap_persist;
  });
}

int ddamg_level_info(ddamg_handle* h, int level, int dims[4], int* ndof, int* ntv) {
  return guard([&] {
    Level& L = level_of(h, level);
    if (dims)
      for (int d = 0; d < 4; ++d) dims[d] = L.g.L[d];
    if (ndof) *ndof = L.n;
    if (ntv) *ntv = L.N;
  });
}

int ddamg_apply(ddamg_handle* h, int level, int precision, const double* in, double* out, int n) {
  return guard([&] {
    Level& L = level_of(h, level);
    if (n < 1 || !in || !out) fail(DDAMG_ERR_ARG, "invalid fields");
    if (precision == 2) {   // double-FP32 arithmetic on FP64 vectors (fine level)
      if (!L.fine) fail(DDAMG_ERR_ARG, "double-FP32 application is on the fine level only");
      if (!L.Udf) df_refresh(h);
      hook<double>(h, level, in, out, n, false, level, [&](cplx<double>* o, cplx<double>* i) {
        Prof pr(h, DDAMG_PROF_FINE_DSLASH, (double)L.vlen * 16 * n * 2 + (double)L.g.V * (36 * 16 + 72 * 8));
        fine_dslash_df(o, i, nullptr, L.Udf, L.clovdf, L.g, L.f64.bc_t, n, L.vlen, h->st);
      });
    } else if (fp32_compute(precision)) {
      hook<float>(h, level, in, out, n, false, level,
                  [&](cplx<float>* o, cplx<float>* i) { apply_D<float>(h, L, o, i, nullptr, n); });
    } else {
      hook<double>(h, level, in, out, n, false, level,
                   [&](cplx<double>* o, cplx<double>* i) { apply_D<double>(h, L, o, i, nullptr, n); });
    }
  });
}

int ddamg_smooth(ddamg_handle* h, int level, int precision, const double* b, double* z, int n, int iterations) {
  return guard([&] {
    Level& L = level_of(h, level);
    if (L.coarsest || n < 1 || !b || !z) fail(DDAMG_ERR_ARG, "no smoother on this level");
    if (fp32_compute(precision))
      hook<float>(h, level, b, z, n, true, level,
                  [&](cplx<float>* o, cplx<float>* i) { sap<float>(h, L, o, i, n, iterations); });
    else
      hook<double>(h, level, b, z, n, true, level,
                   [&](cplx<double>* o, cplx<double>* i) { sap<double>(h, L, o, i, n, iterations); });
  });
}

int ddamg_restrict(ddamg_handle* h, int level, int precision, const double* fine, double* coarse, int n) {
  return guard([&] {
    Level& L = level_of(h, level);
    if (L.coarsest || n < 1) fail(DDAMG_ERR_ARG, "no restriction from the coarsest level");
    if (fp32_compute(precision))
      hook<float>(h, level, fine, coarse, n, false, level + 1,
                  [&](cplx<float>* o, cplx<float>* i) { restrict_lv<float>(h, level, o, i, n); });
    else
      hook<double>(h, level, fine, coarse, n, false, level + 1,
                   [&](cplx<double>* o, cplx<double>* i) { restrict_lv<double>(h, level, o, i, n); });
  });
}

int ddamg_prolong(ddamg_handle* h, int level, int precision, const double* coarse, double* fine, int n) {
  return guard([&] {
    Level& L = level_of(h, level);
    if (L.coarsest || n < 1) fail(DDAMG_ERR_ARG, "no prolongation to the coarsest level");
    if (fp32_compute(precision))
      hook<float>(h, level + 1, coarse, fine, n, false, level,
                  [&](cplx<float>* o, cplx<float>* i) { prolong_lv<float>(h, level, o, i, n, false); });
    else
      hook<double>(h, level + 1, coarse, fine, n, false, level,
                   [&](cplx<double>* o, cplx<double>* i) { prolong_lv<double>(h, level, o, i, n, false); });
  });
}

int ddamg_kcycle(ddamg_handle* h, int level, int precision, const double* b, double* z, int n) {
  return guard([&] {
    Level& L = level_of(h, level);
    if (L.coarsest || n < 1 || n > h->max_batch) fail(DDAMG_ERR_ARG, "K-cycle needs a non-coarsest level, n <= max_rhs");
    if (fp32_compute(precision))
      hook<float>(h, level, b, z, n, false, level,
                  [&](cplx<float>* o, cplx<float>* i) { kcycle_run<float>(h, level, o, i, n); });
    else
      hook<double>(h, level, b, z, n, false, level,
                   [&](cplx<double>* o, cplx<double>* i) { kcycle_run<double>(h, level, o, i, n); });
  });
}

int ddamg_coarse_solve(ddamg_handle* h, int precision, const double* b, double* z, int n) {
  return guard([&] {
    if (!h || n < 1 || n > h->max_batch) fail(DDAMG_ERR_ARG, "n must be 1..max_rhs");
    const int l = h->L - 1;
    if (fp32_compute(precision))
      hook<float>(h, l, b, z, n, false, l, [&](cplx<float>* o, cplx<float>* i) { coarse_solve<float>(h, o, i, n); });
    else
      hook<double>(h, l, b, z, n, false, l,
                   [&](cplx<double>* o, cplx<double>* i) { coarse_solve<double>(h, o, i, n); });
  });
}

int ddamg_set_testvectors(ddamg_handle* h, int level, const double* tv, int n) {
  return guard([&] {
    Level& L = level_of(h, level);
    if (L.coarsest || n != L.N || !tv) fail(DDAMG_ERR_ARG, "n must equal n_tv of the level");
    import_fields(h, L, L.tv64, tv, n);
    sync(h);
  });
}

int ddamg_get_testvectors(ddamg_handle* h, int level, double* tv, int n) {
  return guard([&] {
    Level& L = level_of(h, level);
    if (L.coarsest || n != L.N || !tv) fail(DDAMG_ERR_ARG, "n must equal n_tv of the level");
    hook<double>(h, level, nullptr, tv, n, false, level, [&](cplx<double>* o, cplx<double>*) {
      blas_convert<double, double>(o, L.tv64, L.vlen * n, 1, 0, 0, h->st);
    });
  });
}

int ddamg_rebuild(ddamg_handle* h, int level) {
  return guard([&] {
    Level& L = level_of(h, level);
    if (L.coarsest) fail(DDAMG_ERR_ARG, "no interpolation on the coarsest level");
    rebuild(h, level);
  });
}

int ddamg_get_interpolation(ddamg_handle* h, int level, double* P) {
  return guard([&] {
    Level& L = level_of(h, level);
    if (L.coarsest || !P) fail(DDAMG_ERR_ARG, "no interpolation on the coarsest level");
    hook<double>(h, level, nullptr, P, L.N, false, level, [&](cplx<double>* o, cplx<double>*) {
      blas_convert<double, double>(o, L.P64, L.vlen * L.N, 1, 0, 0, h->st);
    });
  });
}

int ddamg_get_coarse_operator(ddamg_handle* h, int level, double* blocks) {
  return guard([&] {
    Level& L = level_of(h, level);
    if (L.fine || !blocks) fail(DDAMG_ERR_ARG, "coarse operators exist on levels >= 1");
    const size_t bytes = sizeof(cplx<double>) * (size_t)L.g.V * 9 * L.n * L.n;
    const bool dev = is_device_ptr(blocks);
    cplx<double>* d = dev ? reinterpret_cast<cplx<double>*>(blocks) : static_cast<cplx<double>*>(scratch(h, 1, bytes));
    coarse_blocks_export(d, L.c64.blk, L.g, L.n, h->st);
    if (!dev) CK(cudaMemcpyAsync(blocks, d, bytes, cudaMemcpyDeviceToHost, h->st));
    sync(h);
  });
}

int ddamg_setup_times(ddamg_handle* h, double* seconds, int n) {
  if (!h || !seconds || n < 0) {
    g_err = "null argument";
    return DDAMG_ERR_ARG;
  }
  for (int i = 0; i < n; ++i) {
    const int l = i / DDAMG_SETUP_KINDS, k = i % DDAMG_SETUP_KINDS;
    seconds[i] = l < DDAMG_MAX_LEVELS ? h->setup_s[l][k] : 0.0;
  }
  return DDAMG_OK;
}

int ddamg_device_bytes(ddamg_handle* h, size_t* bytes) {
  if (!h || !bytes) {
    g_err = "null argument";
    return DDAMG_ERR_ARG;
  }
  *bytes = h->dev_bytes;
  return DDAMG_OK;
}

int ddamg_estimate_bytes(const int dims[4], const ddamg_params* params, size_t* bytes) {
  if (!dims || !params || !bytes) {
    g_err = "null argument";
    return DDAMG_ERR_ARG;
  }
  return guard([&] {
    validate(*params);
    for (int d = 0; d < 4; ++d)
      if (dims[d] <= 0) fail(DDAMG_ERR_ARG, "lattice extents must be positive");
    *bytes = estimate_bytes(dims, *params);
  });
}

int ddamg_server_create(size_t hbm_budget, ddamg_server** out) {
  if (!out) {
    g_err = "null argument";
    return DDAMG_ERR_ARG;
  }
  *out = nullptr;
  ddamg_server* S = new ddamg_server();
  const int rc = guard([&] {
    if (hbm_budget == 0) {
      size_t fr = 0, total = 0;
      CK(cudaMemGetInfo(&fr, &total));
      hbm_budget = total / 10 * 9;
    }
    S->budget = hbm_budget;
  });
  if (rc != DDAMG_OK) {
    delete S;
    return rc;
  }
  *out = S;
  return DDAMG_OK;
}

int ddamg_server_add(ddamg_server* S, ddamg_handle* h, int* hid) {
  if (!S || !h || !hid) {
    g_err = "null argument";
    return DDAMG_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  for (SrvHier* H : S->hs)
    if (H->h == h) {
      g_err = "hierarchy already registered";
      return DDAMG_ERR_ARG;
    }
  if (S->used + h->dev_bytes > S->budget) {
    g_err = "admission refused: the hierarchy's device footprint (" + std::to_string(h->dev_bytes) +
            " bytes) exceeds the server's remaining HBM budget (" + std::to_string(S->budget - S->used) + " bytes)";
    return DDAMG_ERR_ADMISSION;
  }
  SrvHier* H = new SrvHier();
  H->h = h;
  H->bytes = h->dev_bytes;
  S->used += H->bytes;
  S->hs.push_back(H);
  *hid = (int)S->hs.size() - 1;
  H->worker = std::thread(server_worker, S, H);
  return DDAMG_OK;
}

int ddamg_server_submit(ddamg_server* S, int hid, const double* rhs, int n, double tol, long long* id) {
  if (!S || !rhs || !id || n < 1 || !(tol > 0)) {
    g_err = "invalid argument";
    return DDAMG_ERR_ARG;
  }
  SrvHier* H = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (hid < 0 || hid >= (int)S->hs.size() || S->stop) {
      g_err = "unknown hierarchy or server stopping";
      return DDAMG_ERR_ARG;
    }
    H = S->hs[hid];   // SrvHier objects live until ddamg_server_free
  }
  SrvRequest* rq = new SrvRequest();
  const size_t len = H->h->lv[0].vlen * 2 * (size_t)n;
  if (is_device_ptr(rhs)) {
    delete rq;
    g_err = "serving takes right-hand sides in host memory";
    return DDAMG_ERR_ARG;
  }
  rq->hid = hid;
  rq->n = n;
  rq->tol = tol;
  rq->b.assign(rhs, rhs + len);
  rq->x.assign(len, 0.0);
  rq->st.assign(n, ddamg_stats{});
  rq->remaining = n;
  std::lock_guard<std::mutex> lk(S->mu);
  rq->t_submit = now_seconds();
  *id = S->next_id++;
  S->reqs[*id] = rq;
  for (int c = 0; c < n; ++c) H->queue.emplace_back(rq, c);
  S->work_cv.notify_all();
  return DDAMG_OK;
}

int ddamg_server_poll(ddamg_server* S, long long id, int* done) {
  if (!S || !done) {
    g_err = "null argument";
    return DDAMG_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) {
    g_err = "unknown request";
    return DDAMG_ERR_ARG;
  }
  *done = it->second->status <= 0;
  return DDAMG_OK;
}

int ddamg_server_wait(ddamg_server* S, long long id, double* x, ddamg_stats* per_rhs, double* times) {
  if (!S || !x) {
    g_err = "null argument";
    return DDAMG_ERR_ARG;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) {
    g_err = "unknown request";
    return DDAMG_ERR_ARG;
  }
  SrvRequest* rq = it->second;
  S->done_cv.wait(lk, [&] { return rq->status <= 0; });
  std::memcpy(x, rq->x.data(), sizeof(double) * rq->x.size());
  if (per_rhs)
    for (int c = 0; c < rq->n; ++c) per_rhs[c] = rq->st[c];
  if (times) {
    times[0] = rq->t_start - rq->t_submit;   // queueing before the first restart cycle
    times[1] = rq->t_done - rq->t_submit;    // latency
    times[2] = rq->t_done - rq->t_start;     // time in the batch
  }
  const int rc = rq->status;
  const std::string msg = rq->err;
  S->reqs.erase(it);
  delete rq;
  if (rc != DDAMG_OK)
    g_err = rc == DDAMG_ERR_NOCONV ? std::string("outer FGMRES did not reach the tolerance")
                                   : "request failed: " + (msg.empty() ? std::string("(no message)") : msg);
  return rc;
}

int ddamg_server_free(ddamg_server* S) {
  if (!S) return DDAMG_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->work_cv.notify_all();
  }
  for (SrvHier* H : S->hs) {
    if (H->worker.joinable()) H->worker.join();
    delete H;
  }
  for (auto& kv : S->reqs) delete kv.second;
  delete S;
  return DDAMG_OK;
}

}  // extern "C"
