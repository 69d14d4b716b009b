// libmgiga: handle, device data, V-cycle and PCG drivers, and the C ABI
// declared in include/mgiga.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mgiga.h"
#include "host_problem.hpp"
#include "device.cuh"
#include "host.hpp"
#include "kernels.h"
#include "matfree.hpp"
#include "setup_gpu.hpp"
#include "tune.hpp"

using namespace mgiga;
using namespace mgiga::dev;

namespace {

struct CudaError : std::runtime_error {
  explicit CudaError(const std::string& m) : std::runtime_error(m) {}
};

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      throw CudaError(std::string(#call) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

// Device allocations of one handle; every buffer is freed in the destructor.
// Uploads and fills are ordered on the handle's stream: set-up in one thread
// must not touch the legacy default stream while another thread captures.
struct Arena {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  size_t budget = 0;
  cudaStream_t stream = nullptr;
  ~Arena() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <class T>
  T* alloc(size_t n) {
    if (n == 0) n = 1;
    const size_t b = n * sizeof(T);
    if (budget && bytes + b > budget) throw SetupError(MGIGA_ENOMEM, "device footprint exceeds hbm_budget");
    void* p = nullptr;
    const cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      if (e == cudaErrorMemoryAllocation) throw SetupError(MGIGA_ENOMEM, "cudaMalloc failed: out of device memory");
      throw CudaError(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    ptrs.push_back(p);
    bytes += b;
    return static_cast<T*>(p);
  }
  template <class T>
  T* upload(const std::vector<T>& v) {
    T* p = alloc<T>(v.size());
    if (!v.empty()) CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, stream));
    return p;
  }
  // vector with a zero guard of g elements on both sides; returns the data start
  double* guarded(int64_t n, int64_t g) {
    double* p = alloc<double>((size_t)(n + 2 * g));
    CK(cudaMemsetAsync(p, 0, (size_t)(n + 2 * g) * sizeof(double), stream));
    return p + g;
  }
};

struct DLevel {
  int64_t nloc = 0, guard = 0;
  int ndof = 0, K = 0;
  double *u = nullptr, *f = nullptr, *r = nullptr;
  double* band = nullptr;
  PatchMeta* patches = nullptr;
  Tile* tiles = nullptr;
  int ntiles = 0;
  int nx = 0;
  int64_t* x_row = nullptr;
  int* x_ptr = nullptr;
  int64_t* x_col = nullptr;
  double* x_val = nullptr;
  int nsh = 0;
  int* sh_ptr = nullptr;
  int64_t* sh_pos = nullptr;
  int* sh_patch = nullptr;
  double* weight = nullptr;  // null for SIPG (all copies have weight 1)
  int* loc2glob = nullptr;
  int64_t* owner = nullptr;
  // transfer from level-1 (this level is the fine one)
  XferMeta* xm = nullptr;
  int* par_start = nullptr;
  double* par_val = nullptr;
  int pw = 0;
  int* ch_start = nullptr;
  double* ch_val = nullptr;
  int cw = 0;
  // mode-wise 2D transfers: row blocks of the coarse (restriction) / fine (prolongation) level
  int4* xr_blocks = nullptr;
  int xr_n = 0, xr_smem = 0;
  int4* xp_blocks = nullptr;
  int xp_n = 0, xp_smem = 0;
  int res_g = 0;  // threads per row group of the FP32 cycle residual (0: the built-in rule)
  // fast diagonalisation: GEMM steps
  GemmTask* fd_tasks = nullptr;
  GemmItem* fd_items = nullptr;
  std::vector<std::pair<int, int>> fd_steps;  // item range per step
  std::vector<int> fd_step_ta;                 // element type of A per step (0 double, 1 float)
  int fd_kind = 0;                             // contraction engine: 0 FP64 SIMT, 1 FP32 SIMT, 2 TF32, 3 BF16
  float* r32 = nullptr;                        // FP32 copy of r for the TF32 contractions
  float* rc = nullptr;                         // 2D TF32: compact FP32 interiors of r (16-byte rows)
  int rc_n = 0;
  int64_t rc_total = 0;
  int64_t *rc_eptr = nullptr, *rc_ibase = nullptr, *rc_off = nullptr;
  int *rc_n0 = nullptr, *rc_N0 = nullptr, *rc_ld = nullptr;
  FdFusedTask* fd_fused[2] = {nullptr, nullptr};  // 2D TF32: two chained-contraction passes
  int fd_fused_n[2] = {0, 0};
  int fd_fused_smem = 0;
  FdSmall* fd_small = nullptr;                 // fused path (small 2D patches): one CTA per patch
  int fd_small_n = 0, fd_small_smem = 0;
  FdSmall* fd_cluster = nullptr;               // fused path (2D, FP32): one thread-block cluster per patch
  int fd_cluster_n = 0;
  FdClusterShape fd_cshape{};
  // pieces (interface pieces on levels >= 1, the coarse solve on level 0)
  PieceMeta* pieces = nullptr;
  PieceItem* piece_items = nullptr;
  int npiece_items = 0, piece_max_n = 0;
  void* zpool = nullptr;         // dense inverses: double, or float (zpool_f32) for the pieces of the mixed path
  bool zpool_f32 = false;
  int64_t* piece_pos = nullptr;
  // Gauss-Seidel
  int64_t* gs_pos = nullptr;
  int* gs_patch = nullptr;
  int* gs_cls = nullptr;
  int* gs_x = nullptr;
  double* gs_band = nullptr;  // band rows of the owner copies in colour order
  float* band32 = nullptr;    // FP32 band (mixed path): residuals inside the cycle
  int* gs_cptr_d = nullptr;
  int gs_blocks = 0, gs_blocks_tail = 0;  // cooperative grid: all colours / the colours after the base ones
  std::vector<int> gs_cptr;
  int arith = 0;              // smoother arithmetic: 0 FP64, 1 FP32, 2 FP32 + TF32 tensor-core FD,
                              // 3 FP32 + BF16 tensor-core FD
  int2* gs_stride = nullptr;
  int2* gs_xrange = nullptr;
  int64_t* gs_xcol = nullptr;  // per entry (gs_xrange): SIPG couplings, then further copies' band rows
  double* gs_xval = nullptr;
  // mixed path: base colours of each patch parity swept patch-parallel
  // (staged colour blocks, see gs_patch_staged)
  int gs_base = 0;                 // (p+1)^d base colours per parity
  int gs_csize = 0;                // CTAs per patch cluster (0: grid-wide sweep only)
  int gs_smem = 0;                 // shared memory per CTA of the patch phase
  int* gs_phase_patches[2] = {nullptr, nullptr};
  int gs_nphase[2] = {0, 0};
  GsStagedArgs gs_staged{};        // everything but colours, direction, u
  unsigned char* gs_pool = nullptr;
  int64_t* gs_foff = nullptr;      // byte offset of each entry's f in the pool (-1: none)
  int* gs_xent[2] = {nullptr, nullptr};  // per phase: base-colour entries with couplings to the other parity
  int gs_nxent[2] = {0, 0};
  // matrix-free residual of the finest level (option matrix_free)
  bool mf = false;
  MfDev mfd;
  double mf_flops = 0.0, mf_bytes = 0.0;
  int mf_nx = 0;  // stored couplings: SIPG cross-patch and within-patch terms, CSR over rows
  int64_t* mf_x_row = nullptr;
  int* mf_x_ptr = nullptr;
  int64_t* mf_x_col = nullptr;
  double* mf_x_val = nullptr;
};

}  // namespace

struct mgiga_handle {
  Problem pr;
  mgiga_options opt{};
  int levels = 0;
  std::vector<Level> L;
  std::vector<Transfer> T;
  std::vector<std::vector<int>> colours;   // per level (GS)
  std::vector<std::vector<Piece>> pieces;  // per level (SCMS)
  std::vector<std::vector<int>> piece_of;  // per level (SCMS)
  std::vector<int> num_pieces;
  bool assembled = false;
  std::string err;
  cudaStream_t stream = nullptr;
  int device = -1;          // the CUDA device current at mgiga_assemble (owns every buffer)
  bool own_stream = false;  // created by the library when the options give none
  cudaEvent_t legacy_done = nullptr;  // orders an owned stream after the legacy default stream
  // the smoother's interface-piece solves run beside its fast diagonalisation (disjoint unknowns,
  // both read only r): a second stream of the stream's priority, forked and joined by events
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  std::unique_ptr<Arena> arena;
  std::vector<DLevel> D;
  // PCG state
  double *x = nullptr, *p = nullptr, *q = nullptr, *b = nullptr, *t = nullptr;
  double* scal = nullptr;
  double* partials = nullptr;
  unsigned int* counter = nullptr;
  unsigned int* gs_bar = nullptr;  // grid barrier state of the Gauss-Seidel sweep
  int* gs_err = nullptr;           // set by a kernel whose bounded wait gave up
  long long* probe_ns = nullptr;   // duration of the wait-expiry check
  double *in1 = nullptr, *in2 = nullptr, *out = nullptr;  // staging (global order)
  double* host_scal = nullptr;                            // pinned
  cudaGraphExec_t g_iter_a = nullptr, g_iter_b = nullptr, g_vcycle = nullptr;
  long long g_iter_a_kernels = 0, g_iter_b_kernels = 0;
  // device-driven PCG: the whole iteration loop as one graph with conditional nodes (a while loop
  // around the first half of an iteration, an if for the confirming true residual and one for the
  // second half), steered by control kernels; 0: not built yet, 1: built, -1: unavailable
  cudaGraphExec_t g_solve = nullptr;
  int device_loop = 0;
  CgLoopState* loop_state = nullptr;
  double* dhist = nullptr;
  CgLoopState* host_state = nullptr;  // pinned
  long long g_conf_kernels = 0, g_start_kernels = 0, g_go_kernels = 0;
  cudaGraph_t g_solve_tmpl = nullptr;  // the solve graph (for batch graphs)
  bool pending = false;                // a solve graph was launched and not yet finished
  long long launches = 0;  // kernels enqueued on the device by this handle
  std::vector<double> history;  // relative residuals of the last solve: initial, then per iteration

  ~mgiga_handle() {
    if (g_solve) cudaGraphExecDestroy(g_solve);
    if (g_solve_tmpl) cudaGraphDestroy(g_solve_tmpl);
    if (host_state) cudaFreeHost(host_state);
    if (g_iter_a) cudaGraphExecDestroy(g_iter_a);
    if (g_iter_b) cudaGraphExecDestroy(g_iter_b);
    if (g_vcycle) cudaGraphExecDestroy(g_vcycle);
    if (host_scal) cudaFreeHost(host_scal);
    arena.reset();
    if (own_stream && stream) cudaStreamDestroy(stream);
    if (legacy_done) cudaEventDestroy(legacy_done);
    if (side) cudaStreamDestroy(side);
    if (fork_ev) cudaEventDestroy(fork_ev);
    if (join_ev) cudaEventDestroy(join_ev);
  }
};

namespace {

// ---------------------------------------------------------------------------
// device construction
// ---------------------------------------------------------------------------
std::vector<Tile> make_tiles(const Level& L) {
  std::vector<Tile> t;
  for (int k = 0; k < L.K; ++k)
    for (int64_t s = L.off[k]; s < L.off[k + 1]; s += kTile) {
      Tile x;
      x.patch = k;
      x.start = s;
      x.count = (int)std::min<int64_t>(kTile, L.off[k + 1] - s);
      t.push_back(x);
    }
  return t;
}

int64_t guard_of(const Level& L) {
  int64_t g = 0;
  for (int k = 0; k < L.K; ++k) {
    int64_t s = 0;
    for (int a = 0; a < L.d; ++a) s += L.p * L.stride(k, a);
    g = std::max(g, s);
  }
  return g + 8;
}

void build_transfer_tables(const Level& C, const Level& F, const Transfer& T, Arena& A, DLevel& dl) {
  std::vector<XferMeta> xm(F.K * 3);
  int pw = 1, cw = 1;
  for (int k = 0; k < F.K; ++k)
    for (int a = 0; a < F.d; ++a) {
      const int nf = F.N[k][a], nc = C.N[k][a];
      const Vec& P = T.P[k][a];
      for (int i = 0; i < nf; ++i) {
        int lo = nc, hi = -1;
        for (int I = 0; I < nc; ++I)
          if (P[(size_t)i * nc + I] != 0.0) { lo = std::min(lo, I); hi = std::max(hi, I); }
        if (hi >= lo) pw = std::max(pw, hi - lo + 1);
      }
      for (int I = 0; I < nc; ++I) {
        int lo = nf, hi = -1;
        for (int i = 0; i < nf; ++i)
          if (P[(size_t)i * nc + I] != 0.0) { lo = std::min(lo, i); hi = std::max(hi, i); }
        if (hi >= lo) cw = std::max(cw, hi - lo + 1);
      }
    }
  std::vector<int> ps, cs;
  Vec pv, cv;
  for (int k = 0; k < F.K; ++k)
    for (int a = 0; a < 3; ++a) {
      XferMeta& m = xm[k * 3 + a];
      m.par_off = (int64_t)ps.size();
      m.ch_off = (int64_t)cs.size();
      if (a >= F.d) { m.nf = m.nc = 1; continue; }
      const int nf = F.N[k][a], nc = C.N[k][a];
      m.nf = nf;
      m.nc = nc;
      const Vec& P = T.P[k][a];
      for (int i = 0; i < nf; ++i) {
        int lo = 0;
        while (lo < nc && P[(size_t)i * nc + lo] == 0.0) ++lo;
        if (lo == nc) lo = 0;
        ps.push_back(lo);
        for (int t = 0; t < pw; ++t) pv.push_back(lo + t < nc ? P[(size_t)i * nc + lo + t] : 0.0);
      }
      for (int I = 0; I < nc; ++I) {
        int lo = 0;
        while (lo < nf && P[(size_t)lo * nc + I] == 0.0) ++lo;
        if (lo == nf) lo = 0;
        cs.push_back(lo);
        for (int t = 0; t < cw; ++t) cv.push_back(lo + t < nf ? P[(size_t)(lo + t) * nc + I] : 0.0);
      }
    }
  // 2D: row blocks of the mode-wise kernels, as many output rows (at most 4 coarse / 8 fine: enough
  // CTAs for every SM) as keep the intermediate of the xi_0 pass within 32 KB (FP64), unless
  // MGIGA_XFER_MW=0
  const char* mw_env = std::getenv("MGIGA_XFER_MW");
  if (F.d == 2 && !(mw_env && mw_env[0] == '0')) {
    constexpr int kRowsR = 4, kRowsP = 8, kTarget = 32 * 1024;
    std::vector<int4> rb, pb;
    int rs = 0, pss = 0;
    bool fits = true;
    for (int k = 0; k < F.K && fits; ++k) {
      const XferMeta& m0 = xm[k * 3];
      const XferMeta& m1 = xm[k * 3 + 1];
      const int N1f = F.N[k][1], N1c = C.N[k][1], N0f = F.N[k][0], N0c = C.N[k][0];
      (void)m0;
      auto span_r = [&](int a, int b) {  // fine rows spanned by the children of coarse rows [a, b)
        return std::min(N1f, cs[m1.ch_off + b - 1] + cw) - cs[m1.ch_off + a];
      };
      auto span_p = [&](int a, int b) {  // coarse rows spanned by the parents of fine rows [a, b)
        return std::min(N1c, ps[m1.par_off + b - 1] + pw) - ps[m1.par_off + a];
      };
      for (int a = 0; a < N1c;) {
        int b = a + 1;
        while (b < N1c && b - a < kRowsR && (int64_t)span_r(a, b + 1) * N0c * 8 <= kTarget) ++b;
        const int bytes = span_r(a, b) * N0c * 8;
        if (bytes > kXferSmemMax) fits = false;
        rs = std::max(rs, bytes);
        rb.push_back(make_int4(k, a, b, 0));
        a = b;
      }
      for (int a = 0; a < N1f;) {
        int b = a + 1;
        while (b < N1f && b - a < kRowsP && (int64_t)span_p(a, b + 1) * N0f * 8 <= kTarget) ++b;
        const int bytes = span_p(a, b) * N0f * 8;
        if (bytes > kXferSmemMax) fits = false;
        pss = std::max(pss, bytes);
        pb.push_back(make_int4(k, a, b, 0));
        a = b;
      }
    }
    if (fits) {
      CK(prepare_transfers_mw2());
      dl.xr_blocks = A.upload(rb);
      dl.xr_n = (int)rb.size();
      dl.xr_smem = rs;
      dl.xp_blocks = A.upload(pb);
      dl.xp_n = (int)pb.size();
      dl.xp_smem = pss;
    }
  }
  dl.xm = A.upload(xm);
  dl.par_start = A.upload(ps);
  dl.par_val = A.upload(pv);
  dl.pw = pw;
  dl.ch_start = A.upload(cs);
  dl.ch_val = A.upload(cv);
  dl.cw = cw;
}

// interior fast diagonalisation as batched GEMM steps (Sec. 5 smoother on patch interiors)
// engine: -1 the built-in rule; 0 the batched SIMT contractions; 1 the tensor cores (TF32 / BF16
// modes); 2 the one-CTA-per-patch contractions (2D, when every interior fits shared memory)
// MGIGA_FD_CLUSTER=1: the one-cluster-per-patch fast diagonalisation on 2D FP32 levels (built-in
// rule and autotuner candidate)
bool fd_cluster_opted_in() {
  const char* env = std::getenv("MGIGA_FD_CLUSTER");
  return env && env[0] == '1';
}

void build_fd(const Level& L, int lvl, double delta, double tau, Arena& A, DLevel& dl, int engine = -1) {
  const int d = L.d;
  std::vector<FDData> fd(L.K);
#pragma omp parallel for schedule(dynamic)
  for (int k = 0; k < L.K; ++k) fd[k] = fd_setup(L, k, delta);
  // contraction engine of this level: the tensor cores (TF32 / BF16 modes) only for large
  // interiors; below ~160 per direction the 128 x 64 tiles leave too few CTAs and the 64 x 64 FP32
  // SIMT tiles are faster (measured on the SIPG 3x3 layout)
  int max_n = 0;
  for (int k = 0; k < L.K; ++k)
    for (int a = 0; a < d; ++a) max_n = std::max(max_n, fd[k].n[a]);
  int tensor_min_n = 160;
  if (const char* env = std::getenv("MGIGA_FD_TENSOR_MIN_N")) tensor_min_n = std::max(1, std::atoi(env));
  const int fdk = engine == 1 ? dl.arith
                : engine >= 0 ? (dl.arith <= 1 ? dl.arith : 1)
                : dl.arith <= 1 ? dl.arith : (max_n >= tensor_min_n ? dl.arith : 1);
  dl.fd_kind = fdk;
  // U pool
  Vec Upool;
  std::vector<std::array<int64_t, 3>> uoff(L.K);
  int64_t tsize = 0;
  std::vector<int64_t> toff(L.K);
  for (int k = 0; k < L.K; ++k) {
    int64_t sz = 1;
    for (int a = 0; a < d; ++a) {
      uoff[k][a] = (int64_t)Upool.size();
      Upool.insert(Upool.end(), fd[k].U[a].begin(), fd[k].U[a].end());
      sz *= fd[k].n[a];
    }
    toff[k] = tsize;
    tsize += sz;
  }
  // FP64 path: U and the temporaries in double; FP32 path: in float (the
  // input r and the updated u stay double, converted on load / store)
  const bool f32 = dl.arith >= 1;
  const size_t esz = f32 ? sizeof(float) : sizeof(double);
  char* dU;
  if (f32) {
    std::vector<float> Uf(Upool.begin(), Upool.end());
    dU = reinterpret_cast<char*>(A.upload(Uf));
  } else {
    dU = reinterpret_cast<char*>(A.upload(Upool));
  }
  // inverse eigenvalue sums 1 / (sigma + lambda_{d-1}[i_{d-1}] + .. + lambda_0[i_0]) in interior flat
  // order (i_0 fastest), in the arithmetic type
  Vec dinv((size_t)std::max<int64_t>(tsize, 1), 0.0);
#pragma omp parallel for schedule(dynamic)
  for (int k = 0; k < L.K; ++k) {
    const int n0 = fd[k].n[0], n1 = fd[k].n[1], n2 = d == 3 ? fd[k].n[2] : 1;
    for (int i2 = 0; i2 < n2; ++i2)
      for (int i1 = 0; i1 < n1; ++i1)
        for (int i0 = 0; i0 < n0; ++i0) {
          double den = d == 2 ? fd[k].sigma + fd[k].lam[1][i1] + fd[k].lam[0][i0]
                              : fd[k].sigma + fd[k].lam[2][i2] + fd[k].lam[0][i0] + fd[k].lam[1][i1];
          dinv[(size_t)toff[k] + ((size_t)i2 * n1 + i1) * n0 + i0] = 1.0 / den;
        }
  }
  char* dD;
  if (f32) {
    std::vector<float> df(dinv.begin(), dinv.end());
    dD = reinterpret_cast<char*>(A.upload(df));
  } else {
    dD = reinterpret_cast<char*>(A.upload(dinv));
  }
  char* T1 = reinterpret_cast<char*>(A.alloc<double>((size_t)std::max<int64_t>(tsize, 1)));
  char* T2 = reinterpret_cast<char*>(A.alloc<double>((size_t)std::max<int64_t>(tsize, 1)));
  const int tU = f32 ? 1 : 0;
  // TF32 path: every operand FP32 in memory (the residual copied to FP32 before the first step)
  float* r32 = nullptr;
  if (fdk == 2 && d == 3) {
    r32 = A.alloc<float>((size_t)L.nloc + 8);
    dl.r32 = r32;
  }
  std::vector<GemmTask> tasks;
  std::vector<GemmItem> items;
  dl.fd_steps.clear();
  dl.fd_step_ta.clear();
  auto add_step = [&](const std::vector<GemmTask>& st) {
    const int i0 = (int)items.size();
    dl.fd_step_ta.push_back(st.empty() ? 0 : st[0].tA);  // one element type per step
    for (const auto& g : st) {
      const int id = (int)tasks.size();
      tasks.push_back(g);
      const int bm = fdk >= 2 ? 128 : gemm_tile(fdk);  // tensor-core tiles are 128 x 64
      const int bn = fdk >= 2 ? 64 : bm;
      const int tm = (g.M + bm - 1) / bm, tn = (g.N + bn - 1) / bn;
      for (int z = 0; z < g.batch; ++z)
        for (int a = 0; a < tm; ++a)
          for (int b = 0; b < tn; ++b) items.push_back({id, z, a, b});
    }
    dl.fd_steps.push_back({i0, (int)items.size()});
  };
  auto base = [](GemmTask g) {
    g.transA = g.transB = 0;
    g.batch = 1;
    g.epi = 0;
    g.nhi = 0;
    g.sA = g.sB = g.sC = 0;
    g.alpha = 1.0;
    g.dinv = nullptr;
    g.ldd = 0;
    g.tA = g.tB = g.tC = 0;
    g.vec = g.ctrans = 0;
    return g;
  };
  const int nsteps = d == 2 ? 4 : 6;
  // TF32 in 2D: every operand K-major with rows padded to a multiple of 4 floats (16-byte copies):
  // transposed copies of U_0 and U_1, the outputs of steps 1 and 3 stored transposed, and the
  // residual's interiors gathered into compact FP32 blocks before the first step
  const bool vec2d = fdk == 2 && d == 2;
  auto ld4 = [](int n) { return (n + 3) / 4 * 4; };
  std::vector<std::array<int64_t, 4>> voff(L.K);  // U0, U0^T, U1, U1^T in the vec pool
  std::vector<std::array<int64_t, 4>> toffv(L.K);  // Rc, C1^T, X, Y^T in the temporary pool
  float* vU = nullptr;
  float* vT = nullptr;
  if (vec2d) {
    std::vector<float> pool;
    int64_t tsz = 0;
    for (int k = 0; k < L.K; ++k) {
      const int n0 = fd[k].n[0], n1 = fd[k].n[1];
      auto put = [&](const Vec& U, int n, bool transpose) {
        const int64_t off = (int64_t)pool.size();
        pool.resize(pool.size() + (size_t)n * ld4(n), 0.0f);
        for (int i = 0; i < n; ++i)
          for (int j = 0; j < n; ++j)
            pool[off + (size_t)i * ld4(n) + j] = (float)(transpose ? U[(size_t)j * n + i] : U[(size_t)i * n + j]);
        return off;
      };
      voff[k] = {put(fd[k].U[0], n0, false), put(fd[k].U[0], n0, true), put(fd[k].U[1], n1, false),
                 put(fd[k].U[1], n1, true)};
      toffv[k][0] = tsz; tsz += (int64_t)n1 * ld4(n0);  // Rc: n1 x n0
      toffv[k][1] = tsz; tsz += (int64_t)n0 * ld4(n1);  // C1^T: n0 x n1
      toffv[k][2] = tsz; tsz += (int64_t)n1 * ld4(n0);  // X: n1 x n0
      toffv[k][3] = tsz; tsz += (int64_t)n0 * ld4(n1);  // Y^T: n0 x n1
    }
    vU = A.upload(pool);
    vT = A.alloc<float>((size_t)std::max<int64_t>(tsz, 4));
    CK(cudaMemsetAsync(vT, 0, (size_t)std::max<int64_t>(tsz, 4) * sizeof(float), A.stream));  // padding columns stay 0
    std::vector<int64_t> e_ptr(1, 0), ib, doff;
    std::vector<int> n0s, N0s, dld;
    for (int k = 0; k < L.K; ++k) {
      const int n0 = fd[k].n[0], n1 = fd[k].n[1];
      e_ptr.push_back(e_ptr.back() + (int64_t)n0 * n1);
      ib.push_back(L.off[k] + 1 + L.N[k][0]);
      n0s.push_back(std::max(n0, 1));
      N0s.push_back(L.N[k][0]);
      doff.push_back(toffv[k][0]);
      dld.push_back(ld4(n0));
    }
    dl.rc = vT;
    dl.rc_n = L.K;
    dl.rc_total = e_ptr.back();
    dl.rc_eptr = A.upload(e_ptr);
    dl.rc_ibase = A.upload(ib);
    dl.rc_n0 = A.upload(n0s);
    dl.rc_N0 = A.upload(N0s);
    dl.rc_off = A.upload(doff);
    dl.rc_ld = A.upload(dld);
  }
  std::vector<std::vector<GemmTask>> steps(nsteps);
  for (int k = 0; k < L.K; ++k) {
    const int n0 = fd[k].n[0], n1 = fd[k].n[1], n2 = d == 3 ? fd[k].n[2] : 1;
    if (n0 <= 0 || n1 <= 0 || n2 <= 0) continue;
    const int64_t N0 = L.N[k][0], N01 = (int64_t)L.N[k][0] * L.N[k][1];
    const int64_t ibase = L.off[k] + 1 + N0 + (d == 3 ? N01 : 0);  // interior (1,1[,1])
    const void* U0 = dU + uoff[k][0] * esz;
    const void* U1 = dU + uoff[k][1] * esz;
    const void* U2 = d == 3 ? dU + uoff[k][2] * esz : nullptr;
    void* Tk = T1 + toff[k] * esz;
    void* Xk = T2 + toff[k] * esz;
    const void* Dk = dD + toff[k] * esz;
    GemmTask g{};
    // element types: U and temporaries tU; r (first input) and u (last output) double
    auto types = [&](GemmTask& t, int ta, int tb, int tc) { t.tA = ta; t.tB = tb; t.tC = tc; };
    if (vec2d) {
      const float* U0v = vU + voff[k][0];
      const float* U0t = vU + voff[k][1];
      const float* U1v = vU + voff[k][2];
      const float* U1t = vU + voff[k][3];
      float* Rc = vT + toffv[k][0];
      float* C1t = vT + toffv[k][1];
      float* Xv = vT + toffv[k][2];
      float* Yt = vT + toffv[k][3];
      auto vtask = [&](GemmTask t) { t.vec = 1; t.transA = 0; t.transB = 1; t.tA = t.tB = 1; return t; };
      // 1) C1 = R U0, stored transposed
      g = base(g); g.M = n1; g.N = n0; g.K = n0; g.A = Rc; g.lda = ld4(n0); g.B = U0t; g.ldb = ld4(n0);
      g.C = C1t; g.ldc = ld4(n1); g.ctrans = 1; g.ndiv = n0; g.tC = 1; steps[0].push_back(vtask(g));
      // 2) X = (U1^T C1) * dinv
      g = base(g); g.M = n1; g.N = n0; g.K = n1; g.A = U1t; g.lda = ld4(n1); g.B = C1t; g.ldb = ld4(n1);
      g.C = Xv; g.ldc = ld4(n0); g.ndiv = n0; g.epi = 1; g.dinv = Dk; g.ldd = n0; g.tC = 1;
      steps[1].push_back(vtask(g));
      // 3) Y = X U0^T, stored transposed
      g = base(g); g.M = n1; g.N = n0; g.K = n0; g.A = Xv; g.lda = ld4(n0); g.B = U0v; g.ldb = ld4(n0);
      g.C = Yt; g.ldc = ld4(n1); g.ctrans = 1; g.ndiv = n0; g.tC = 1; steps[2].push_back(vtask(g));
      // 4) u_interior += tau U1 Y
      g = base(g); g.M = n1; g.N = n0; g.K = n1; g.A = U1v; g.lda = ld4(n1); g.B = Yt; g.ldb = ld4(n1);
      g.C = dl.u + ibase; g.ldc = N0; g.ndiv = n0; g.epi = 2; g.alpha = tau; g.tC = 0;
      steps[3].push_back(vtask(g));
    } else if (d == 2) {
      // 1) T = R U0   (R: n1 x n0 rows of the interior, ld N0; its FP32 copy on the TF32 path)
      g = base(g); g.M = n1; g.N = n0; g.K = n0; g.lda = N0; g.B = U0; g.ldb = n0;
      if (r32) { g.A = r32 + ibase; types(g, 1, tU, tU); } else { g.A = dl.r + ibase; types(g, 0, tU, tU); }
      g.C = Tk; g.ldc = n0; g.ndiv = n0; steps[0].push_back(g);
      // 2) X = U1^T T, divided by lambda1[m] + lambda0[n] + sigma
      g = base(g); g.M = n1; g.N = n0; g.K = n1; g.A = U1; g.transA = 1; g.lda = n1; g.B = Tk; g.ldb = n0;
      g.C = Xk; g.ldc = n0; g.ndiv = n0; g.epi = 1; g.dinv = Dk; g.ldd = n0; types(g, tU, tU, tU);
      steps[1].push_back(g);
      // 3) Y1 = X U0^T
      g = base(g); g.M = n1; g.N = n0; g.K = n0; g.A = Xk; g.lda = n0; g.B = U0; g.transB = 1; g.ldb = n0;
      g.C = Tk; g.ldc = n0; g.ndiv = n0; types(g, tU, tU, tU); steps[2].push_back(g);
      // 4) u_interior += tau U1 Y1
      g = base(g); g.M = n1; g.N = n0; g.K = n1; g.A = U1; g.lda = n1; g.B = Tk; g.ldb = n0;
      g.C = dl.u + ibase; g.ldc = N0; g.ndiv = n0; g.epi = 2; g.alpha = tau; types(g, tU, tU, 0); steps[3].push_back(g);
    } else {
      const int64_t plane = (int64_t)n1 * n0;
      // 1) T[i2] = R[i2] U0  (batched over planes i2)
      g = base(g); g.M = n1; g.N = n0; g.K = n0; g.lda = N0; g.sA = N01; g.B = U0; g.ldb = n0;
      if (r32) { g.A = r32 + ibase; types(g, 1, tU, tU); } else { g.A = dl.r + ibase; types(g, 0, tU, tU); }
      g.C = Tk; g.ldc = n0; g.sC = plane; g.ndiv = n0; g.batch = n2; steps[0].push_back(g);
      // 2) X[i2] = U1^T T[i2]
      g = base(g); g.M = n1; g.N = n0; g.K = n1; g.A = U1; g.transA = 1; g.lda = n1; g.B = Tk; g.ldb = n0;
      g.sB = plane; g.C = Xk; g.ldc = n0; g.sC = plane; g.ndiv = n0; g.batch = n2; types(g, tU, tU, tU); steps[1].push_back(g);
      // 3) T = U2^T X  (n2 x n1 n0), divided by the eigenvalue sums
      g = base(g); g.M = n2; g.N = (int)plane; g.K = n2; g.A = U2; g.transA = 1; g.lda = n2; g.B = Xk; g.ldb = plane;
      g.C = Tk; g.ldc = plane; g.ndiv = (int)plane; g.epi = 1; g.dinv = Dk; g.ldd = plane; types(g, tU, tU, tU);
      steps[2].push_back(g);
      // 4) X = T U0^T  (n2 n1 x n0)
      g = base(g); g.M = n2 * n1; g.N = n0; g.K = n0; g.A = Tk; g.lda = n0; g.B = U0; g.transB = 1; g.ldb = n0;
      g.C = Xk; g.ldc = n0; g.ndiv = n0; types(g, tU, tU, tU); steps[3].push_back(g);
      // 5) T[j2] = U1 X[j2]
      g = base(g); g.M = n1; g.N = n0; g.K = n1; g.A = U1; g.lda = n1; g.B = Xk; g.ldb = n0; g.sB = plane;
      g.C = Tk; g.ldc = n0; g.sC = plane; g.ndiv = n0; g.batch = n2; types(g, tU, tU, tU); steps[4].push_back(g);
      // 6) u_interior += tau U2 T  (columns (i1, i0) -> i1 N0 + i0)
      g = base(g); g.M = n2; g.N = (int)plane; g.K = n2; g.A = U2; g.lda = n2; g.B = Tk; g.ldb = plane;
      g.C = dl.u + ibase; g.ldc = N01; g.ndiv = n0; g.nhi = N0; g.epi = 2; g.alpha = tau; types(g, tU, tU, 0); steps[5].push_back(g);
    }
  }
  for (auto& s : steps) add_step(s);
  (void)lvl;
  // 2D TF32 with MGIGA_FD_CHAINED=1: the four steps as two launches of chained contractions
  // (fd_fused_tf32), when every interior fits the kernel's tensor memory.  Not the default: on the
  // benchmark layout its 16-wide K slabs, each behind a CTA barrier and an MMA-completion wait, make
  // it latency-bound (finest level, p = 6: 0.130 ms against 0.091 ms for the four separate steps)
  const char* chained_env = std::getenv("MGIGA_FD_CHAINED");
  if (vec2d && chained_env && chained_env[0] == '1' && engine <= 1) {
    bool fits = true;
    for (int k = 0; k < L.K; ++k) fits = fits && fd[k].n[1] <= fd_fused_max_rows();
    if (fits) {
      std::vector<FdFusedTask> ft[2];
      int mt_max = 1;
      for (int k = 0; k < L.K; ++k) {
        const int n0 = fd[k].n[0], n1 = fd[k].n[1];
        if (n0 <= 0 || n1 <= 0) continue;
        const int mt = (n1 + 127) / 128, nb = (n0 + 31) / 32;
        mt_max = std::max(mt_max, mt);
        for (int pass = 0; pass < 2; ++pass)
          for (int rb = 0; rb < mt; ++rb)
            for (int cb = 0; cb < nb; ++cb) {
              FdFusedTask q{};
              q.n0 = n0;
              q.n1 = n1;
              q.rb = rb;
              q.cb = cb;
              q.mt = mt;
              q.pass = pass;
              q.ldr = ld4(n0);
              q.ldb = ld4(n0);
              q.ldl = ld4(n1);
              q.ldx = ld4(n0);
              q.N0 = L.N[k][0];
              q.ibase = L.off[k] + 1 + L.N[k][0];
              if (pass == 0) {  // T = R U_0[:, cb], X = (U_1^T T) dinv
                q.rin = vT + toffv[k][0];
                q.bt = vU + voff[k][1];
                q.lm = vU + voff[k][3];
                q.dinv = reinterpret_cast<const float*>(dD) + toff[k];
                q.xout = vT + toffv[k][2];
              } else {  // T = X U_0^T[:, cb], u += tau U_1 T
                q.rin = vT + toffv[k][2];
                q.bt = vU + voff[k][0];
                q.lm = vU + voff[k][2];
                q.u = dl.u;
              }
              ft[pass].push_back(q);
            }
      }
      CK(prepare_fd_fused());
      for (int pass = 0; pass < 2; ++pass) {
        dl.fd_fused[pass] = A.upload(ft[pass]);
        dl.fd_fused_n[pass] = (int)ft[pass].size();
      }
      dl.fd_fused_smem = fd_fused_smem(mt_max);
    }
  }
  if (fdk <= 1) CK(prepare_gemm());
  // small 2D interiors: all four contractions of a patch in one CTA (shared memory), unless
  // MGIGA_FD_FUSE=0 (kept for testing the batched-GEMM path on small problems)
  const char* fuse_env = std::getenv("MGIGA_FD_FUSE");
  int fuse_max_n = 48;
  if (const char* env = std::getenv("MGIGA_FD_FUSE_MAX_N")) fuse_max_n = std::max(1, std::atoi(env));
  if (engine == 2) fuse_max_n = 1 << 30;  // forced: whatever fits shared memory
  // 2D interiors on the FP32 path: all four contractions of a patch by one thread-block cluster
  // (engine 3), with MGIGA_FD_CLUSTER=1 wherever it fits.  Opt-in: measured on the SIPG 3x3 layout,
  // p = 6, one solve alone it is faster (interiors of 52-76: 0.047 -> 0.021 ms, 28-40: 0.023 ->
  // 0.013 ms; V-cycle 2.59 -> 2.57 ms, p = 2 1.40 -> 1.34 ms), but five solves side by side ran 2.5%
  // slower (its clusters of 8-16 CTAs wait for whole SMs that the other solves' kernels hold)
  const bool cl_off = fuse_env && fuse_env[0] == '0';
  if (d == 2 && f32 && !cl_off && (engine == 3 || (engine < 0 && fd_cluster_opted_in() && fdk == 1))) {
    std::vector<FdSmall> fc;
    int n0max = 0, n1max = 0;
    for (int k = 0; k < L.K; ++k) {
      const int n0 = fd[k].n[0], n1 = fd[k].n[1];
      if (n0 <= 0 || n1 <= 0) continue;
      n0max = std::max(n0max, n0);
      n1max = std::max(n1max, n1);
      FdSmall q{};
      q.ibase = L.off[k] + 1 + L.N[k][0];
      q.n0 = n0;
      q.n1 = n1;
      q.N0 = L.N[k][0];
      q.U0 = dU + uoff[k][0] * esz;
      q.U1 = dU + uoff[k][1] * esz;
      q.dinv = dD + toff[k] * esz;
      fc.push_back(q);
    }
    FdClusterShape sh{};
    if (!fc.empty() && fd_cluster_shape(n0max, n1max, (int)fc.size(), &sh)) {
      dl.fd_cluster = A.upload(fc);
      dl.fd_cluster_n = (int)fc.size();
      dl.fd_cshape = sh;
    }
  }
  if (d == 2 && !(fuse_env && fuse_env[0] == '0') && engine != 0 && engine != 1 && engine != 3 && !dl.fd_cluster) {
    std::vector<FdSmall> fs;
    int smem = 0;
    bool fits = true;
    for (int k = 0; k < L.K && fits; ++k) {
      const int n0 = fd[k].n[0], n1 = fd[k].n[1];
      if (n0 <= 0 || n1 <= 0) continue;
      const int b = fd_small_smem(n0, n1, f32);
      // one CTA does 4 n^3 multiply-adds: beyond n = 48 the batched steps over all SMs win
      // (measured on the SIPG 3x3 layout: n ~ 30-45 fused 0.023 ms vs 0.039; n ~ 60-93 0.062 vs 0.048)
      if (b > kFdSmallSmem || std::max(n0, n1) > fuse_max_n) { fits = false; break; }
      smem = std::max(smem, b);
      FdSmall q{};
      q.ibase = L.off[k] + 1 + L.N[k][0];
      q.n0 = n0;
      q.n1 = n1;
      q.N0 = L.N[k][0];
      q.U0 = dU + uoff[k][0] * esz;
      q.U1 = dU + uoff[k][1] * esz;
      q.dinv = dD + toff[k] * esz;
      fs.push_back(q);
    }
    if (fits && !fs.empty()) {
      CK(prepare_fd_small());
      dl.fd_small = A.upload(fs);
      dl.fd_small_n = (int)fs.size();
      dl.fd_small_smem = smem;
    }
  }
  dl.fd_tasks = A.upload(tasks);
  dl.fd_items = A.upload(items);
}

void build_pieces(const std::vector<Piece>& pcs, const Level& L, Arena& A, DLevel& dl, bool coarse) {
  std::vector<PieceMeta> meta;
  std::vector<PieceItem> items;
  std::vector<int64_t> pos;
  std::vector<Vec> Z;
  std::vector<const Piece*> use;
  for (const auto& pc : pcs)
    if (coarse || pc.kind == 1) use.push_back(&pc);
  Z.resize(use.size());
  int err = 0;
  std::string msg;
  // small pieces side by side, large ones one at a time with the threads inside the factorisation
  constexpr int kLargePiece = 1024;
#pragma omp parallel for schedule(dynamic)
  for (int i = 0; i < (int)use.size(); ++i) {
    if ((int)use[i]->dofs.size() >= kLargePiece) continue;
    try {
      Z[i] = spd_inverse(restrict_dense(L, use[i]->dofs), (int)use[i]->dofs.size());
    } catch (const SetupError& e) {
#pragma omp critical
      { err = e.status; msg = e.what(); }
    }
  }
  for (int i = 0; i < (int)use.size() && !err; ++i) {
    if ((int)use[i]->dofs.size() < kLargePiece) continue;
    try {
      Z[i] = spd_inverse(restrict_dense(L, use[i]->dofs), (int)use[i]->dofs.size(), true);
    } catch (const SetupError& e) {
      err = e.status;
      msg = e.what();
    }
  }
  if (err) throw SetupError(err, msg);
  int64_t zoff = 0;
  Vec zpool;
  int maxn = 0;
  for (size_t i = 0; i < use.size(); ++i) {
    PieceMeta m;
    m.n = (int)use[i]->dofs.size();
    m.z_off = zoff;
    m.dof_off = (int64_t)pos.size();
    m.pad = 0;
    for (int g : use[i]->dofs) pos.push_back(L.owner[g]);
    zpool.insert(zpool.end(), Z[i].begin(), Z[i].end());
    zoff += (int64_t)m.n * m.n;
    maxn = std::max(maxn, m.n);
    for (int r0 = 0; r0 < m.n; r0 += 64) items.push_back({(int)meta.size(), r0});
    meta.push_back(m);
  }
  dl.pieces = A.upload(meta);
  dl.piece_items = A.upload(items);
  dl.npiece_items = (int)items.size();
  dl.piece_max_n = maxn;
  // the coarse solve stays FP64; the interface pieces of the mixed-precision smoother run in FP32
  dl.zpool_f32 = !coarse && dl.arith >= 1;
  if (dl.zpool_f32) {
    std::vector<float> zf(zpool.begin(), zpool.end());
    dl.zpool = A.upload(zf);
  } else {
    dl.zpool = A.upload(zpool);
  }
  dl.piece_pos = A.upload(pos);
  if (maxn > 0) CK(prepare_piece_kernel(maxn));
}

// Colour blocks of the staged patch-parallel sweep (mixed path).  A group is
// (base colour c, patch k, slab r of the patch's cluster); its rows are split
// into as few items as keep two item buffers in shared memory, each item a
// block of float coef[line][Rp][2p+1] (line: the band offsets along the slower
// directions; a row's 2p+1 coefficients along xi_0 contiguous, so one thread
// reads them at fixed offsets), int lidx[Rp] ((slow index - slab start) << 20 |
// index in the plane), float f[Rp] (f minus the couplings to the other parity,
// written before each phase) and float dinv[Rp] (1 / diagonal), padded to 16
// bytes.  Rp >= rows and the shared-memory pitch of a slow index are chosen so
// that the threads of a warp read distinct banks.  Items are ordered by
// (phase, k, r, colour, item); runs of consecutive items (in sweep order) that
// fit one buffer are fetched as one chunk.
void build_gs_staged(const Problem& pr, const std::vector<int>& colour, const Level& L, Arena& A, DLevel& dl,
                     const std::vector<int>& order, const std::vector<int64_t>& gpos, const std::vector<int>& gpatch,
                     const std::vector<int>& gx, int ncol, int B, int gs_cluster) {
  auto gxr_of = [&](int e) { return gx[e] >= 0 && L.x_ptr[gx[e] + 1] > L.x_ptr[gx[e]]; };
  const int K = L.K, d = L.d, nb = L.nb, P = L.p;
  const int W = 2 * P + 1, nob = d == 2 ? W : W * W;
  const int center = d == 2 ? P * W + P : (P * W + P) * W + P;
  const int nbase = std::min(ncol, 2 * B);
  const int nent = nbase > 0 ? dl.gs_cptr[nbase] : 0;
  if (nent == 0) return;
  auto plane_of = [&](int k) { return d == 2 ? (int64_t)L.N[k][0] : (int64_t)L.N[k][0] * L.N[k][1]; };
  auto nslow_of = [&](int k) { return L.N[k][d - 1]; };
  std::vector<int> cls_of(L.ndof, -1);
  for (size_t c = 0; c + 1 < L.sh_ptr.size(); ++c) cls_of[L.loc2glob[L.sh_pos[L.sh_ptr[c]]]] = (int)c;
  for (int e = 0; e < nent; ++e)
    if (cls_of[order[e]] >= 0) throw SetupError(MGIGA_EINVAL, "shared DoF on a base colour");
  for (int k = 0; k < K; ++k)
    if (plane_of(k) >= (1 << 20) || nslow_of(k) >= (1 << 11)) return;  // beyond the packed index: grid-wide sweep
  // most lanes of one warp that hit one bank (a warp: 32 / tpr rows spaced p + 1 apart, tpr coefficient lines)
  auto bank_degree = [&](int tpr, auto word) {
    int cnt[32] = {0}, worst = 0;
    for (int j = 0; j < 32 / tpr; ++j)
      for (int q = 0; q < std::min(tpr, nob); ++q) worst = std::max(worst, ++cnt[((word(j, q) % 32) + 32) % 32]);
    return worst;
  };
  int64_t limit = 225 * 1024;
  if (const char* env = std::getenv("MGIGA_GS_SMEM_KB")) {  // tuning: leave room for other streams' CTAs
    const int v = std::atoi(env);
    if (v >= 48 && v <= 225) limit = (int64_t)v * 1024;
  }
  auto item_bytes = [&](int rp) { return ((int64_t)(nb + 3) * rp * 4 + 15) / 16 * 16; };
  // buffers of the streamed (non-resident) case
  int ring = kGsRing;
  if (const char* env = std::getenv("MGIGA_GS_NBUF")) {  // tuning
    const int v = std::atoi(env);
    if (v >= 2 && v <= kGsRingMax) ring = v;
  }
  struct Plan {
    int cs = 0, threads = 0, tpr = 0, nbuf = 0, max_items = 0;
    int64_t cap = 0, total = 0;
    int off_buf = 0, off_mbar = 0, off_meta = 0;
    std::vector<int> slab, pitch, guard, grp_of, rows, nsub, rp_deg;
    int rp_best = 0;
    int rp_of(int x) const {  // padded rows: smallest Rp >= x with the fewest bank conflicts
      if (x <= 0) return 0;
      while (rp_deg[x % 32] != rp_best) ++x;
      return x;
    }
  };
  auto plan_for = [&](int cs, Plan& pl) -> bool {
    pl.cs = cs;
    pl.slab.resize(K);
    for (int k = 0; k < K; ++k) pl.slab[k] = (nslow_of(k) + cs - 1) / cs;
    const int ngrp = nbase * K * cs;
    pl.grp_of.assign(nent, 0);
    pl.rows.assign(ngrp, 0);
    for (int e = 0; e < nent; ++e) {
      const int c = colour[order[e]], k = gpatch[e];
      const int r = (int)((gpos[e] - L.off[k]) / plane_of(k)) / pl.slab[k];
      const int g = (c * K + k) * cs + r;
      pl.grp_of[e] = g;
      pl.rows[g]++;
    }
    int max_rows = 0;
    for (int v : pl.rows) max_rows = std::max(max_rows, v);
    // CTA shape: a row is summed by tpr threads (its coefficient lines split
    // among them, then a shuffle tree), threads / tpr rows at a time; minimise
    // the dependent steps of the longest colour plus the cycles its warp
    // instructions take on the SM's four schedulers (per warp and line 3 W:
    // two loads and an FMA per coefficient; per warp and pass ~50 for the
    // row's set-up and update).  Measured on the finest level at p = 6
    // (16-CTA clusters): 512 x 4 0.194 ms, 1024 x 4 0.201, 512 x 8 0.206,
    // 1024 x 8 0.210, 256 x 4 0.213, 1024 x 16 0.237 -- the order this cost gives.
    double best = 1e30;
    for (int nt : {256, 512, 1024})
      for (int tpr : {4, 8, 16, 32}) {
        const int passes = std::max(1, (max_rows + nt / tpr - 1) / (nt / tpr));
        const int lines = (nob + tpr - 1) / tpr;
        const double latency = passes * (lines * (W * 2.0 + 40.0) + 40.0 * std::log2((double)tpr)) + nt / 8.0;
        const double issue =
            (double)max_rows * tpr / 32.0 * (lines * 3.0 * W + 6.0 * std::log2((double)tpr) + 50.0) / 4.0;
        const double cost = latency + issue;
        if (cost < best) {
          best = cost;
          pl.threads = nt;
          pl.tpr = tpr;
        }
      }
    if (const char* env = std::getenv("MGIGA_GS_SHAPE")) {  // "threads,tpr": manual override for tuning
      int nt = 0, tp = 0;
      if (std::sscanf(env, "%d,%d", &nt, &tp) == 2 && (nt == 256 || nt == 512 || nt == 1024) &&
          (tp == 4 || tp == 8 || tp == 16 || tp == 32)) {
        pl.threads = nt;
        pl.tpr = tp;
      }
    }
    const int tpr = pl.tpr;
    // padded rows: coefficient line q of row j starts at word (q Rp + j) W
    pl.rp_deg.assign(32, 0);
    pl.rp_best = 1 << 30;
    for (int x = 0; x < 32; ++x) {
      pl.rp_deg[x] = bank_degree(tpr, [&](int j, int q) { return (q * x + j) * W; });
      pl.rp_best = std::min(pl.rp_best, pl.rp_deg[x]);
    }
    // slab pitch and guards; the extended slab
    int64_t ext = 0;
    pl.pitch.resize(K);
    pl.guard.resize(K);
    for (int k = 0; k < K; ++k) {
      const int plane = (int)plane_of(k), N0 = L.N[k][0];
      int bp = plane, bd = 1 << 30;
      for (int x = plane; x < plane + 32; ++x) {
        const int dg = bank_degree(tpr, [&](int j, int q) {
          return (P + 1) * j + (d == 2 ? q * x : (q % W) * N0 + (q / W) * x);
        });
        if (dg < bd) { bd = dg; bp = x; }
      }
      pl.pitch[k] = bp;
      pl.guard[k] = ((d == 2 ? P : P * N0 + P) + 3) / 4 * 4;
      ext = std::max<int64_t>(ext, 2 * pl.guard[k] + (int64_t)(pl.slab[k] + 2 * P) * bp);
    }
    pl.off_buf = (int)((ext * 4 + 127) / 128 * 128);
    // whole phase regions resident (one buffer, no splitting) if they fit
    std::vector<int64_t> region((size_t)2 * K * cs, 0);
    for (int g = 0; g < ngrp; ++g) {
      const int c = g / (K * cs), kr = g % (K * cs);
      region[(size_t)(c / B) * K * cs + kr] += item_bytes(pl.rp_of(pl.rows[g]));
    }
    int64_t max_region = 0;
    for (int64_t v : region) max_region = std::max(max_region, v);
    pl.nsub.assign(ngrp, 1);
    const int64_t resident_room = limit - pl.off_buf - 16 - 32 * (int64_t)B;
    if (max_region <= resident_room) {
      pl.nbuf = 1;
      pl.cap = (max_region + 15) / 16 * 16;
      pl.max_items = B;
    } else {
      // a ring of nbuf buffers, nbuf - 1 chunks in flight while one is read;
      // groups larger than a buffer split into near-equal items
      pl.nbuf = ring;
      const int64_t mbar_room = (8 * (int64_t)ring + 15) / 16 * 16;
      for (int extra = 1; extra <= 8; extra *= 2) {  // meta room for up to extra x B items
        const int64_t cap = (limit - pl.off_buf - mbar_room - 32 * (int64_t)B * extra) / ring / 16 * 16;
        int rmax = 0;
        while (item_bytes(pl.rp_of(rmax + 1)) <= cap) ++rmax;
        if (rmax < 1) return false;
        std::vector<int> items((size_t)2 * K * cs, 0);
        for (int g = 0; g < ngrp; ++g) {
          pl.nsub[g] = std::max(1, (pl.rows[g] + rmax - 1) / rmax);
          const int c = g / (K * cs), kr = g % (K * cs);
          items[(size_t)(c / B) * K * cs + kr] += pl.nsub[g];
        }
        int mi = 0;
        for (int v : items) mi = std::max(mi, v);
        if (mi <= extra * B) {
          pl.cap = cap;
          pl.max_items = mi;
          break;
        }
      }
      if (pl.cap == 0) return false;
    }
    pl.off_mbar = (int)((pl.off_buf + pl.nbuf * pl.cap + 15) / 16 * 16);
    pl.off_meta = pl.off_mbar + (8 * pl.nbuf + 15) / 16 * 16;
    pl.total = pl.off_meta + 32 * (int64_t)pl.max_items;
    return pl.total <= limit;
  };
  // cluster size: the largest (16 CTAs, slabs of a patch side by side) once a
  // colour holds >= 64 rows of a patch, else one CTA per patch (the CTA barrier
  // is cheaper than the cluster barrier and the colour's work is small);
  // measured on the SIPG 3x3 layout, p = 2..6, all levels
  int maxrows_pk = 1;
  {
    std::vector<int> cnt((size_t)nbase * K, 0);
    for (int e = 0; e < nent; ++e) cnt[(size_t)colour[order[e]] * K + gpatch[e]]++;
    for (int v : cnt) maxrows_pk = std::max(maxrows_pk, v);
  }
  const int large = (gs_cluster == 2 || gs_cluster == 4 || gs_cluster == 8) ? gs_cluster : 16;
  std::vector<int> sizes = maxrows_pk >= 64 ? std::vector<int>{large, 16, 8, 4, 2, 1} : std::vector<int>{1, 2, 4, 8, 16};
  if (const char* env = std::getenv("MGIGA_GS_CS")) {  // manual cluster size for tuning
    const int v = std::atoi(env);
    if (v == 1 || v == 2 || v == 4 || v == 8 || v == 16) sizes.insert(sizes.begin(), v);
  }
  dl.gs_csize = 0;
  Plan pl;
  for (int cs : sizes) {
    Plan t;
    if (!plan_for(cs, t) || !gs_staged_fits(d, P, t.tpr, cs, (int)t.total, t.threads)) continue;
    pl = std::move(t);
    dl.gs_csize = cs;
    dl.gs_smem = (int)pl.total;
    break;
  }
  if (dl.gs_csize == 0) return;  // the grid-wide sweep handles every colour
  const int cs = dl.gs_csize;
  // items in (phase, k, r, colour, item) order; an item takes a contiguous share of its group's rows
  const int ngrp = nbase * K * cs;
  std::vector<std::vector<int>> members(ngrp);
  for (int e = 0; e < nent; ++e) members[pl.grp_of[e]].push_back(e);
  std::vector<int> sub_ptr(ngrp + 1, 0);
  for (int g = 0; g < ngrp; ++g) sub_ptr[g + 1] = sub_ptr[g] + pl.nsub[g];
  const int nitems_all = sub_ptr[ngrp];
  std::vector<int> it_r0(nitems_all), it_rows(nitems_all), it_rp(nitems_all);
  std::vector<int64_t> it_off(nitems_all, 0), it_bytes(nitems_all, 0);
  for (int g = 0; g < ngrp; ++g)
    for (int j = 0; j < pl.nsub[g]; ++j) {
      const int i = sub_ptr[g] + j, R = pl.rows[g];
      it_r0[i] = (int)((int64_t)R * j / pl.nsub[g]);
      it_rows[i] = (int)((int64_t)R * (j + 1) / pl.nsub[g]) - it_r0[i];
      it_rp[i] = pl.rp_of(it_rows[i]);
      it_bytes[i] = it_rows[i] > 0 ? item_bytes(it_rp[i]) : 0;
    }
  int64_t total = 0;
  for (int ph = 0; ph < 2; ++ph)
    for (int k = 0; k < K; ++k)
      for (int r = 0; r < cs; ++r)
        for (int c = ph * B; c < std::min((ph + 1) * B, nbase); ++c) {
          const int g = (c * K + k) * cs + r;
          for (int i = sub_ptr[g]; i < sub_ptr[g + 1]; ++i) {
            it_off[i] = total;
            total += it_bytes[i];
          }
        }
  std::vector<unsigned char> pool((size_t)std::max<int64_t>(total, 16), 0);
  std::vector<int64_t> foff(L.ndof, -1);
  // groups write disjoint parts of the pool (and of foff): in parallel
#pragma omp parallel for schedule(dynamic, 4)
  for (int g = 0; g < ngrp; ++g) {
    const int k = (g / cs) % K, r = g % cs;
    const int64_t plane = plane_of(k);
    for (int i = sub_ptr[g]; i < sub_ptr[g + 1]; ++i) {
      const int R = it_rows[i], Rp = it_rp[i];
      if (R == 0) continue;
      float* coef = reinterpret_cast<float*>(pool.data() + it_off[i]);
      int* lidx = reinterpret_cast<int*>(coef + (size_t)nb * Rp);
      float* fv = reinterpret_cast<float*>(lidx + Rp);
      float* dinv = fv + Rp;
      for (int row = 0; row < R; ++row) {
        const int e = members[g][it_r0[i] + row];
        const int64_t pos = gpos[e];
        for (int ob = 0; ob < nob; ++ob)
          for (int o0 = 0; o0 < W; ++o0)
            coef[((size_t)ob * Rp + row) * W + o0] = (float)L.band[(size_t)(ob * W + o0) * L.nloc + pos];
        const int64_t loc = pos - L.off[k];
        const int s = (int)(loc / plane), rest = (int)(loc % plane);
        lidx[row] = ((s - r * pl.slab[k]) << 20) | rest;
        dinv[row] = (float)(1.0 / L.band[(size_t)center * L.nloc + pos]);
        foff[e] = it_off[i] + ((int64_t)nb + 1) * Rp * 4 + (int64_t)row * 4;
      }
    }
  }
  // A base colour fixes every index modulo p + 1 (the slow one outermost), so
  // the rows of a run of colours with one residue rho of the slow index read
  // only their own slow index among those = rho (mod p + 1) within reach P:
  // during such a run no CTA reads a halo value a neighbour updates, nor
  // updates one a neighbour reads.  The cluster barrier (halo exchange) is
  // needed only where the residue changes; between the colours of a run the
  // CTA barrier orders the CTA's own slab.
  const int run_len = B % (P + 1) == 0 ? B / (P + 1) : 1;
  auto slow_residue = [&](int c) { return (c % B) / run_len; };
  // per (direction, phase, k, r): items in sweep order grouped into chunks
  const size_t nreg = (size_t)2 * 2 * K * cs;
  std::vector<int64_t> item_ptr(nreg + 1, 0);
  std::vector<int4> cmeta, chunks;
  cmeta.reserve((size_t)2 * nitems_all);
  chunks.reserve((size_t)2 * nitems_all);
  for (int dir = 0; dir < 2; ++dir)
    for (int ph = 0; ph < 2; ++ph)
      for (int k = 0; k < K; ++k)
        for (int r = 0; r < cs; ++r) {
          const size_t reg = (((size_t)dir * 2 + ph) * K + k) * cs + r;
          const int c0 = ph * B, nc = std::max(0, std::min((ph + 1) * B, nbase) - c0);
          // items in sweep order; the last item of each colour flagged (1), and
          // of each run of colours with one residue of the slow index (2)
          std::vector<int> seq;
          std::vector<char> last;
          for (int ci = 0; ci < nc; ++ci) {
            const int c = dir == 0 ? c0 + ci : c0 + nc - 1 - ci;
            const int g = (c * K + k) * cs + r;
            const int n_i = sub_ptr[g + 1] - sub_ptr[g];
            const bool run_end = ci == nc - 1 || slow_residue(c) != slow_residue(dir == 0 ? c + 1 : c - 1);
            for (int j = 0; j < n_i; ++j) {
              seq.push_back(dir == 0 ? sub_ptr[g] + j : sub_ptr[g + 1] - 1 - j);
              last.push_back(j == n_i - 1 ? (run_end ? 3 : 1) : 0);
            }
          }
          std::vector<int> chunk_of(seq.size());
          std::vector<int64_t> lo, hi;
          for (size_t q = 0; q < seq.size(); ++q) {
            const int64_t a0 = it_off[seq[q]], a1 = a0 + it_bytes[seq[q]];
            if (!lo.empty() && std::max(hi.back(), a1) - std::min(lo.back(), a0) <= pl.cap) {
              lo.back() = std::min(lo.back(), a0);
              hi.back() = std::max(hi.back(), a1);
            } else {
              lo.push_back(a0);
              hi.push_back(a1);
            }
            chunk_of[q] = (int)lo.size() - 1;
          }
          item_ptr[reg] = (int64_t)cmeta.size();
          for (size_t q = 0; q < seq.size(); ++q) {
            const int i = seq[q], j = chunk_of[q];
            cmeta.push_back(make_int4(it_rows[i], j, (int)(it_off[i] - lo[j]),
                                      it_rp[i] | ((last[q] & 1) << 30) | ((last[q] >> 1) << 29)));
          }
          for (size_t q = 0; q < seq.size(); ++q)
            chunks.push_back(q < lo.size() ? make_int4((int)(uint32_t)(lo[q] & 0xffffffffLL), (int)(lo[q] >> 32),
                                                       (int)(hi[q] - lo[q]), 0)
                                           : make_int4(0, 0, 0, 0));
          item_ptr[reg + 1] = (int64_t)cmeta.size();
        }
  if (cmeta.empty()) {
    cmeta.push_back(make_int4(0, 0, 0, 0));
    chunks.push_back(make_int4(0, 0, 0, 0));
  }
  dl.gs_pool = A.upload(pool);
  dl.gs_foff = A.upload(foff);
  for (int ph = 0; ph < 2; ++ph) {
    std::vector<int> xe;
    const int e_lo = dl.gs_cptr[std::min(ph * B, nbase)], e_hi = dl.gs_cptr[std::min((ph + 1) * B, nbase)];
    for (int e = e_lo; e < e_hi; ++e)
      if (gxr_of(e)) xe.push_back(e);
    dl.gs_nxent[ph] = (int)xe.size();
    dl.gs_xent[ph] = xe.empty() ? nullptr : A.upload(xe);
  }
  const auto par = patch_parity(pr);
  for (int ph = 0; ph < 2; ++ph) {
    std::vector<int> pp;
    for (int k = 0; k < K; ++k)
      if (par[k] == ph) pp.push_back(k);
    dl.gs_nphase[ph] = (int)pp.size();
    dl.gs_phase_patches[ph] = A.upload(pp);
  }
  GsStagedArgs& a = dl.gs_staged;
  a.K = K;
  a.csize = cs;
  a.base = B;
  a.nbuf = pl.nbuf;
  a.cap = (int)pl.cap;
  a.threads = pl.threads;
  a.tpr = pl.tpr;
  a.slab = A.upload(pl.slab);
  a.pitch = A.upload(pl.pitch);
  a.guard = A.upload(pl.guard);
  a.pool = dl.gs_pool;
  a.item_ptr = A.upload(item_ptr);
  a.cmeta = A.upload(cmeta);
  a.chunks = A.upload(chunks);
  a.max_items = pl.max_items;
  a.off_buf = pl.off_buf;
  a.off_mbar = pl.off_mbar;
  a.off_meta = pl.off_meta;
}

// matrix-free residual of the finest level: point tables, tiling and window partials (matfree.cu),
// and the stored couplings it leaves to CSR: the SIPG cross-patch blocks and the SIPG terms within
// one patch (summed per entry in cell order; rows and columns of Dirichlet positions dropped, as the
// band drops them)
void build_mf(const Problem& pr, const Level& L, const std::vector<std::pair<int64_t, double>>& self, Arena& A,
              DLevel& d) {
  std::string why;
  if (!mf_supported(pr, &why)) throw SetupError(MGIGA_EINVAL, "the matrix-free residual needs " + why);
  const bool f32 = d.arith >= 1;
  const MfHost m = mf_build_host(pr, L, f32);
  auto up = [&](const std::vector<double>& v) -> const void* {
    if (f32) return A.upload(std::vector<float>(v.begin(), v.end()));
    return A.upload(v);
  };
  d.mfd.pp = A.upload(m.pp);
  d.mfd.K = L.K;
  d.mfd.GM = m.GM;
  d.mfd.ntile = m.ntile;
  d.mfd.B = up(m.B);
  d.mfd.Dv = up(m.Dv);
  d.mfd.w = up(m.w);
  d.mfd.gB = up(m.gB);
  d.mfd.gD = up(m.gD);
  d.mfd.ctrl = up(m.ctrl);
  d.mfd.dir = A.upload(L.dirichlet);
  d.mfd.part = f32 ? static_cast<void*>(A.alloc<float>((size_t)m.part_n)) : static_cast<void*>(A.alloc<double>((size_t)m.part_n));
  d.mf_flops = m.flops;
  // u and f read, out written, the window partials written and read back
  d.mf_bytes = 24.0 * (double)L.nloc + 2.0 * (double)m.part_n * (f32 ? 4.0 : 8.0);
  std::map<int64_t, std::vector<std::pair<int64_t, double>>> rows;
  for (size_t i = 0; i < L.x_row.size(); ++i)
    for (int j = L.x_ptr[i]; j < L.x_ptr[i + 1]; ++j) rows[L.x_row[i]].push_back({L.x_col[j], L.x_val[j]});
  // self: one entry per band index (summed in cell order), sorted by index
  for (const auto& x : self) {
    const int64_t o = x.first / L.nloc, r = x.first % L.nloc;
    const int64_t c = r + L.band_offset(L.patch_of[r], (int)o);
    if (L.dirichlet[r] || L.dirichlet[c]) continue;
    rows[r].push_back({c, x.second});
  }
  std::vector<int64_t> xr, xc;
  std::vector<int> xp(1, 0);
  Vec xv;
  for (const auto& r : rows) {
    xr.push_back(r.first);
    for (const auto& e : r.second) {
      xc.push_back(e.first);
      xv.push_back(e.second);
    }
    xp.push_back((int)xc.size());
  }
  d.mf_nx = (int)xr.size();
  d.mf_x_row = A.upload(xr);
  d.mf_x_ptr = A.upload(xp);
  d.mf_x_col = A.upload(xc);
  d.mf_x_val = A.upload(xv);
  d.mf = true;
  if (std::getenv("MGIGA_VERBOSE"))
    std::fprintf(stderr, "mgiga: matrix-free residual: %d tiles of %d^%d elements, %lld partials, %d coupled rows\n",
                 m.ntile, m.te, L.d, (long long)m.part_n, d.mf_nx);
}

void build_gs(const Problem& pr, const std::vector<int>& colour, const Level& L, Arena& A, DLevel& dl,
              int gs_cluster) {
  const int n = L.ndof;
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return colour[a] < colour[b]; });
  std::vector<int> cls_of(n, -1);
  for (size_t c = 0; c + 1 < L.sh_ptr.size(); ++c) cls_of[L.loc2glob[L.sh_pos[L.sh_ptr[c]]]] = (int)c;
  std::vector<int> xr_of_pos;
  std::vector<int64_t> gpos;
  std::vector<int> gpatch, gcls, gx;
  std::unordered_map<int64_t, int> xrow;
  for (size_t i = 0; i < L.x_row.size(); ++i) xrow[L.x_row[i]] = (int)i;
  dl.gs_cptr.assign(1, 0);
  int cur = 0;  // cptr index = colour
  for (int e = 0; e < n; ++e) {
    const int g = order[e];
    while (colour[g] != cur) { dl.gs_cptr.push_back(e); ++cur; }
    const int64_t pos = L.owner[g];
    gpos.push_back(pos);
    gpatch.push_back(L.patch_of[pos]);
    gcls.push_back(cls_of[g]);
    auto it = xrow.find(pos);
    gx.push_back(it == xrow.end() ? -1 : it->second);
  }
  dl.gs_cptr.push_back(n);
  // per entry, the couplings summed besides its own band row: the SIPG couplings of its row, then
  // (conforming) the band rows of the further copies of a shared DoF, whose diagonals are folded
  // into the entry's diagonal (the copies hold the same value); the row's lanes share them
  const int center = L.d == 2 ? L.p * (2 * L.p + 1) + L.p : (L.p * (2 * L.p + 1) + L.p) * (2 * L.p + 1) + L.p;
  std::vector<int2> gst(n), gxr(n);
  std::vector<int64_t> xcol;
  Vec xval, cdiag(n, 0.0);
  for (int e = 0; e < n; ++e) {
    const int k = gpatch[e];
    gst[e] = make_int2(L.N[k][0], L.N[k][0] * L.N[k][1]);
    const int x0 = (int)xcol.size();
    if (gx[e] >= 0)
      for (int j = L.x_ptr[gx[e]]; j < L.x_ptr[gx[e] + 1]; ++j) {
        xcol.push_back(L.x_col[j]);
        xval.push_back(L.x_val[j]);
      }
    if (gcls[e] >= 0)
      for (int cp = L.sh_ptr[gcls[e]] + 1; cp < L.sh_ptr[gcls[e] + 1]; ++cp) {
        const int64_t q = L.sh_pos[cp];
        const int kq = L.patch_of[q];
        for (int o = 0; o < L.nb; ++o) {
          const double v = L.band[(size_t)o * L.nloc + q];
          if (v == 0.0) continue;
          if (o == center) {
            cdiag[e] += v;
          } else {
            xcol.push_back(q + L.band_offset(kq, o));
            xval.push_back(v);
          }
        }
      }
    if (xcol.size() >= (size_t)INT32_MAX) throw SetupError(MGIGA_ENOMEM, "Gauss-Seidel coupling list too long");
    gxr[e] = make_int2(x0, (int)xcol.size());
  }
  // band rows of the owner copies in colour order (coalesced per colour),
  // in double (FP64 path) or float (mixed path)
  const bool f32 = dl.arith >= 1;
  if (f32) {
    std::vector<float> gb((size_t)L.nb * n);
#pragma omp parallel for schedule(static)
    for (int o = 0; o < L.nb; ++o)
      for (int e = 0; e < n; ++e)
        gb[(size_t)o * n + e] = (float)(L.band[(size_t)o * L.nloc + gpos[e]] + (o == center ? cdiag[e] : 0.0));
    dl.gs_band = reinterpret_cast<double*>(A.upload(gb));
  } else {
    Vec gb((size_t)L.nb * n);
#pragma omp parallel for schedule(static)
    for (int o = 0; o < L.nb; ++o)
      for (int e = 0; e < n; ++e) gb[(size_t)o * n + e] = L.band[(size_t)o * L.nloc + gpos[e]] + (o == center ? cdiag[e] : 0.0);
    dl.gs_band = A.upload(gb);
  }
  dl.gs_stride = A.upload(gst);
  dl.gs_xrange = A.upload(gxr);
  dl.gs_xcol = A.upload(xcol);
  dl.gs_xval = A.upload(xval);
  dl.gs_cptr_d = A.upload(dl.gs_cptr);
  const int ncol = (int)dl.gs_cptr.size() - 1;
  int B = 1;
  for (int a = 0; a < L.d; ++a) B *= L.p + 1;
  dl.gs_base = B;
  if (f32) build_gs_staged(pr, colour, L, A, dl, order, gpos, gpatch, gx, ncol, B, gs_cluster);
  int maxrows = 1;
  for (size_t c = 0; c + 1 < dl.gs_cptr.size(); ++c) maxrows = std::max(maxrows, dl.gs_cptr[c + 1] - dl.gs_cptr[c]);
  const int coop = gs_coop_max_blocks(L.d, L.p, f32);
  if (coop <= 0) throw CudaError("cooperative launch not available for the Gauss-Seidel sweep");
  dl.gs_blocks = std::max(1, std::min(coop, (maxrows * 8 + 255) / 256));
  // the colours after the base colours (swept grid-wide after the patch-parallel phases): blocks
  // for their largest colour only (few rows each: a small grid keeps the grid barrier short)
  int maxrows_tail = 1;
  for (size_t c = std::min<size_t>(2 * B, dl.gs_cptr.size() - 1); c + 1 < dl.gs_cptr.size(); ++c)
    maxrows_tail = std::max(maxrows_tail, dl.gs_cptr[c + 1] - dl.gs_cptr[c]);
  dl.gs_blocks_tail = dl.gs_csize > 0 ? std::max(1, std::min(coop, (maxrows_tail * 8 + 255) / 256)) : dl.gs_blocks;
  if (std::getenv("MGIGA_VERBOSE"))
    std::fprintf(stderr,
                 "mgiga: gs level ndof %d colours %d base %d cluster %d smem %d buffers %d x %d bytes threads %d "
                 "tpr %d\n",
                 n, ncol, B, dl.gs_csize, dl.gs_smem, dl.gs_staged.nbuf, dl.gs_staged.cap, dl.gs_staged.threads,
                 dl.gs_staged.tpr);
  dl.gs_pos = A.upload(gpos);
  dl.gs_patch = A.upload(gpatch);
  dl.gs_cls = A.upload(gcls);
  dl.gs_x = A.upload(gx);
}

// ---------------------------------------------------------------------------
// operations on the device (enqueued on h->stream)
// ---------------------------------------------------------------------------
bool conforming(const mgiga_handle* h) { return h->pr.coupling == MGIGA_CONFORMING; }

void residual(mgiga_handle* h, int l, const double* u, const double* f, double* out) {
  const Level& L = h->L[l];
  DLevel& d = h->D[l];
  launch_band(L.d, L.p, 0, d.ntiles, h->stream, d.tiles, d.patches, d.band, d.nloc, u, f, out);
  launch_cross(0, d.nx, h->stream, d.x_row, d.x_ptr, d.x_col, d.x_val, u, out);
  if (conforming(h)) launch_shared(d.nsh, h->stream, d.sh_ptr, d.sh_pos, out, f, 0);
}

// residual inside the cycle: feeds the smoothers and the restriction, so on
// the mixed path the band part runs with FP32 coefficients and arithmetic
void cycle_residual(mgiga_handle* h, int l, const double* u, const double* f, double* out) {
  const Level& L = h->L[l];
  DLevel& d = h->D[l];
  if (d.mf) {  // stiffness by sum factorisation at the Gauss points, stored SIPG couplings
    mf_launch(L.d, L.p, d.arith >= 1, d.mfd, h->stream, u, f, out, d.ntiles, d.tiles);
    launch_cross(0, d.mf_nx, h->stream, d.mf_x_row, d.mf_x_ptr, d.mf_x_col, d.mf_x_val, u, out);
    if (conforming(h)) launch_shared(d.nsh, h->stream, d.sh_ptr, d.sh_pos, out, f, 0);
    return;
  }
  if (!d.band32) {
    residual(h, l, u, f, out);
    return;
  }
  launch_band_residual_f32(L.d, L.p, d.ntiles, h->stream, d.tiles, d.patches, d.band32, d.nloc, u, f, out, d.res_g);
  launch_cross(0, d.nx, h->stream, d.x_row, d.x_ptr, d.x_col, d.x_val, u, out);
  if (conforming(h)) launch_shared(d.nsh, h->stream, d.sh_ptr, d.sh_pos, out, f, 0);
}

void matvec(mgiga_handle* h, int l, const double* u, double* out) {
  const Level& L = h->L[l];
  DLevel& d = h->D[l];
  launch_band(L.d, L.p, 1, d.ntiles, h->stream, d.tiles, d.patches, d.band, d.nloc, u, nullptr, out);
  launch_cross(1, d.nx, h->stream, d.x_row, d.x_ptr, d.x_col, d.x_val, u, out);
  if (conforming(h)) launch_shared(d.nsh, h->stream, d.sh_ptr, d.sh_pos, out, nullptr, 1);
}

// one step of the fast diagonalisation: SIMT tiles (FP64 / FP32) or tensor-core tiles (TF32 / BF16)
void run_fd_step(mgiga_handle* h, DLevel& d, size_t i) {
  const auto& s = d.fd_steps[i];
  if (d.fd_kind == 2)
    launch_gemm_umma_tf32(s.second - s.first, h->stream, d.fd_tasks, d.fd_items + s.first, h->gs_err);
  else if (d.fd_kind == 3)
    launch_gemm_umma(s.second - s.first, 1, h->stream, d.fd_tasks, d.fd_items + s.first, h->gs_err);
  else
    launch_gemm(s.second - s.first, d.fd_kind, d.fd_step_ta[i], h->stream, d.fd_tasks, d.fd_items + s.first);
}

// the interior part of the smoother: fused per patch on small 2D levels, else the batched GEMM steps
void run_fd(mgiga_handle* h, DLevel& d) {
  if (d.fd_cluster) {
    CK(launch_fd_cluster(d.fd_cluster_n, d.fd_cshape, h->stream, d.fd_cluster, d.r, d.u, h->opt.tau));
    return;
  }
  if (d.fd_small) {
    launch_fd_small(d.fd_small_n, d.fd_small_smem, d.arith >= 1, h->stream, d.fd_small, d.r, d.u, h->opt.tau);
    return;
  }
  if (d.r32) launch_to_f32(d.nloc, h->stream, d.r, d.r32);
  if (d.rc)
    launch_gather_interior_f32(d.rc_n, d.rc_total, h->stream, d.rc_eptr, d.rc_ibase, d.rc_n0, d.rc_N0, d.rc_off,
                               d.rc_ld, d.r, d.rc);
  if (d.fd_fused_n[0] > 0) {
    for (int pass = 0; pass < 2; ++pass)
      launch_fd_fused(d.fd_fused_n[pass], d.fd_fused_smem, h->stream, d.fd_fused[pass], h->opt.tau, h->gs_err);
    return;
  }
  for (size_t i = 0; i < d.fd_steps.size(); ++i) run_fd_step(h, d, i);
}

// u += tau sum_T P_T L_T^{-1} P_T^T r  (Eq. Ldef), r in d.r.  The pieces T partition the unknowns
// (patch interiors and interface pieces), so the interface-piece solves and the interiors' fast
// diagonalisation read only r and update disjoint entries of u: the pieces go on the side stream
// (forked from the handle's stream and joined back; under graph capture, two parallel branches)
void smooth(mgiga_handle* h, int l) {
  DLevel& d = h->D[l];
  const bool fork = h->side && d.npiece_items > 0;
  cudaStream_t ps = fork ? h->side : h->stream;
  if (fork) {
    CK(cudaEventRecord(h->fork_ev, h->stream));
    CK(cudaStreamWaitEvent(h->side, h->fork_ev, 0));
  }
  launch_piece(d.npiece_items, d.piece_max_n, ps, d.piece_items, d.pieces, d.zpool, d.zpool_f32, d.piece_pos, d.r, d.u,
               h->opt.tau, 0);
  if (fork) CK(cudaEventRecord(h->join_ev, h->side));
  run_fd(h, d);
  if (fork) CK(cudaStreamWaitEvent(h->stream, h->join_ev, 0));
  if (conforming(h)) launch_shared(d.nsh, h->stream, d.sh_ptr, d.sh_pos, d.u, nullptr, 2);
}

// one Gauss-Seidel sweep: the base colours of each patch parity patch-parallel
// (one launch per parity, a cluster per patch), then the remaining colours
// (DoFs coupling patches of one parity) grid-wide; reversed for the backward sweep
void gs_sweep(mgiga_handle* h, int l, bool forward) {
  const Level& L = h->L[l];
  DLevel& d = h->D[l];
  GsSweepArgs a;
  const int ncol = (int)d.gs_cptr.size() - 1;
  if (ncol <= 0) return;
  a.forward = forward ? 1 : 0;
  a.cptr = d.gs_cptr_d;
  a.ngs = d.ndof;
  a.gsband = d.gs_band;
  a.gs_pos = d.gs_pos; a.gs_stride = d.gs_stride; a.gs_xrange = d.gs_xrange; a.gs_cls = d.gs_cls;
  a.patches = d.patches; a.band = d.band; a.nloc = d.nloc;
  a.sh_ptr = d.sh_ptr; a.sh_pos = d.sh_pos; a.sh_patch = d.sh_patch;
  a.x_col = d.gs_xcol; a.x_val = d.gs_xval; a.f = d.f; a.u = d.u;
  a.bar = h->gs_bar;
  a.err = h->gs_err;
  const bool f32 = d.arith >= 1;
  const int B = d.gs_base;
  auto coop = [&](int cb, int ce, int blocks) {
    a.c_begin = std::min(cb, ncol);
    a.c_end = std::min(ce, ncol);
    if (a.c_end <= a.c_begin) return;
    CK(cudaMemsetAsync(h->gs_bar, 0, 2 * sizeof(unsigned int), h->stream));
    CK(launch_gs_sweep(L.d, L.p, f32, blocks, h->stream, a));
  };
  auto phase = [&](int ph) {
    if (d.gs_csize == 0) {  // no staged plan (FP64 path, or slabs too large): grid-wide sweep
      coop(ph * B, (ph + 1) * B, d.gs_blocks);
      return;
    }
    GsStagedArgs g = d.gs_staged;
    g.c_begin = std::min(ph * B, ncol);
    g.c_end = std::min((ph + 1) * B, ncol);
    if (g.c_end <= g.c_begin) return;
    g.forward = forward ? 1 : 0;
    g.phase_patches = d.gs_phase_patches[ph];
    g.patches = d.patches;
    g.u = d.u;
    g.err = h->gs_err;
    // f minus the couplings to the other parity (fixed during the phase) into the blocks
    const int e0 = d.gs_cptr[g.c_begin], e1 = d.gs_cptr[g.c_end];
    launch_gs_fill_phase(e0, e1 - e0, d.gs_nxent[ph], d.gs_xent[ph], h->stream, d.gs_foff, d.gs_pos, d.gs_xrange,
                         d.gs_xcol, d.gs_xval, d.f, d.u, d.gs_pool);
    CK(launch_gs_staged(L.d, L.p, d.gs_nphase[ph], d.gs_smem, h->stream, g));
  };
  auto tail = [&]() { coop(2 * B, ncol, d.gs_blocks_tail); };
  if (forward) { phase(0); phase(1); tail(); }
  else { tail(); phase(1); phase(0); }
}

// f_{l-1} = P^T r_l (r_l consistent; weights make each shared DoF count once).
// cycle: inside the V-cycle, where the mixed path transfers in FP32 arithmetic
void restrict_to(mgiga_handle* h, int l, const double* r, bool cycle = false) {
  const Level& Lc = h->L[l - 1];
  DLevel& df = h->D[l];
  DLevel& dc = h->D[l - 1];
  if (df.xr_n > 0)
    launch_restrict_mw2(cycle && df.arith >= 1, df.xr_n, df.xr_smem, h->stream, df.xr_blocks, dc.patches, df.patches,
                        df.xm, df.ch_start, df.ch_val, df.cw, r, df.weight, dc.loc2glob, dc.f);
  else
    launch_restrict(Lc.d, cycle && df.arith >= 1, dc.ntiles, h->stream, dc.tiles, dc.patches, df.patches, df.xm,
                    df.ch_start, df.ch_val, df.cw, r, df.weight, dc.loc2glob, dc.f);
  if (conforming(h)) launch_shared(dc.nsh, h->stream, dc.sh_ptr, dc.sh_pos, dc.f, nullptr, 1);
}

void prolong_from(mgiga_handle* h, int l, const double* e, double* u, bool cycle = false) {
  const Level& Lf = h->L[l];
  DLevel& df = h->D[l];
  DLevel& dc = h->D[l - 1];
  if (df.xp_n > 0)
    launch_prolong_mw2(cycle && df.arith >= 1, df.xp_n, df.xp_smem, h->stream, df.xp_blocks, df.patches, dc.patches,
                       df.xm, df.par_start, df.par_val, df.pw, e, u);
  else
    launch_prolong(Lf.d, cycle && df.arith >= 1, df.ntiles, h->stream, df.tiles, df.patches, dc.patches, df.xm,
                   df.par_start, df.par_val, df.pw, e, u);
}

void coarse_solve(mgiga_handle* h) {
  DLevel& d = h->D[0];
  if (d.ndof == 0) {
    CK(cudaMemsetAsync(d.u, 0, d.nloc * sizeof(double), h->stream));
    return;
  }
  launch_piece(d.npiece_items, d.piece_max_n, h->stream, d.piece_items, d.pieces, d.zpool, d.zpool_f32, d.piece_pos, d.f, d.u,
               1.0, 1);
  if (conforming(h)) launch_shared(d.nsh, h->stream, d.sh_ptr, d.sh_pos, d.u, nullptr, 2);
}

// MULTIGRID(l, f_l, 0) of Algorithm 1 / Algorithm 2; result in D[l].u
void vcycle(mgiga_handle* h, int l) {
  if (l == 0) { coarse_solve(h); return; }
  DLevel& d = h->D[l];
  const int sm = h->opt.smoother, nu = h->opt.nu;
  CK(cudaMemsetAsync(d.u, 0, d.nloc * sizeof(double), h->stream));
  bool zero = true;
  if (sm == MGIGA_SMOOTHER_GS || sm == MGIGA_SMOOTHER_HYBRID) {
    const int n = sm == MGIGA_SMOOTHER_GS ? nu : 1;
    for (int i = 0; i < n; ++i) gs_sweep(h, l, true);
    zero = false;
  }
  if (sm == MGIGA_SMOOTHER_SCMS || sm == MGIGA_SMOOTHER_HYBRID) {
    for (int i = 0; i < nu; ++i) {
      if (zero) CK(cudaMemcpyAsync(d.r, d.f, d.nloc * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
      else cycle_residual(h, l, d.u, d.f, d.r);
      smooth(h, l);
      zero = false;
    }
  }
  for (int m = 0; m < std::max(1, h->opt.mu); ++m) {
    cycle_residual(h, l, d.u, d.f, d.r);
    restrict_to(h, l, d.r, true);
    vcycle(h, l - 1);
    prolong_from(h, l, h->D[l - 1].u, d.u, true);
  }
  if (sm == MGIGA_SMOOTHER_SCMS || sm == MGIGA_SMOOTHER_HYBRID) {
    for (int i = 0; i < nu; ++i) {
      cycle_residual(h, l, d.u, d.f, d.r);
      smooth(h, l);
    }
  }
  if (sm == MGIGA_SMOOTHER_GS || sm == MGIGA_SMOOTHER_HYBRID) {
    const int n = sm == MGIGA_SMOOTHER_GS ? nu : 1;
    for (int i = 0; i < n; ++i) gs_sweep(h, l, false);
  }
}

void check_launch() {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw CudaError(std::string("kernel launch: ") + cudaGetErrorString(e));
}

// a Gauss-Seidel sweep whose grid barrier gave up leaves gs_err set; read and
// clear it after the stream has drained
// An owned stream is non-blocking: order it after the legacy default stream,
// on which a caller's device inputs may still be in flight.
void after_legacy(mgiga_handle* h) {
  if (!h->own_stream) return;
  CK(cudaEventRecord(h->legacy_done, cudaStreamLegacy));
  CK(cudaStreamWaitEvent(h->stream, h->legacy_done, 0));
}

void check_device_timeout(mgiga_handle* h) {
  if (!h->gs_err) return;
  int e = 0;
  CK(cudaMemcpyAsync(&e, h->gs_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (e) {
    CK(cudaMemsetAsync(h->gs_err, 0, sizeof(int), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    throw SetupError(MGIGA_ETIMEOUT, "a bounded device wait expired (grid barrier or asynchronous copy)");
  }
}

// adds the kernels enqueued during an API call to the handle's count
struct LaunchScope {
  mgiga_handle* h;
  long long c0;
  explicit LaunchScope(mgiga_handle* hh) : h(hh), c0(launch_counter()) {}
  ~LaunchScope() { h->launches += launch_counter() - c0; }
};

mgiga_status fail(mgiga_handle* h, int st, const std::string& msg) {
  if (h) h->err = msg;
  return (mgiga_status)st;
}

template <class F>
mgiga_status guarded_call(mgiga_handle* h, F&& fn) {
  try {
    return fn();
  } catch (const SetupError& e) {
    return fail(h, e.status, e.what());
  } catch (const CudaError& e) {
    return fail(h, MGIGA_ECUDA, e.what());
  } catch (const std::bad_alloc&) {
    return fail(h, MGIGA_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(h, MGIGA_EINVAL, e.what());
  }
}

// device time (ms) of one application of `fn` on the handle's stream, after one warm-up
template <class F>
double time_on_stream(mgiga_handle* h, F&& fn) {
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  fn();
  CK(cudaEventRecord(a, h->stream));
  fn();
  CK(cudaEventRecord(b, h->stream));
  CK(cudaEventSynchronize(b));
  float ms = 0.0f;
  CK(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  check_launch();
  return ms;
}

// autotuned fast diagonalisation of level l: the contraction engine (batched SIMT tiles, tensor-core
// tiles, one CTA per patch) with the shortest measured application for this size bucket; on a miss
// every candidate is built and timed (the losers' device data stay allocated until mgiga_destroy)
void tune_fd(mgiga_handle* h, const Level& L, int l, Arena& A, DLevel& d, bool verbose) {
  int max_int = 1;
  for (int k = 0; k < L.K; ++k) {
    int64_t v = 1;
    for (int a = 0; a < L.d; ++a) v *= std::max(0, L.N[k][a] - 2);
    max_int = (int)std::max<int64_t>(max_int, v);
  }
  const TuneKey key{TUNE_FD, L.d, L.p, h->opt.precision, tune_bucket(max_int)};
  std::vector<int> cand = {0};
  if (d.arith >= 2) cand.push_back(1);
  if (L.d == 2) cand.push_back(2);
  if (L.d == 2 && d.arith >= 1 && fd_cluster_opted_in()) cand.push_back(3);
  int choice = -1;
  if (!Tuner::instance().lookup(key, &choice)) {
    std::vector<DLevel> built(cand.size(), d);
    choice = Tuner::instance().choose(key, (int)cand.size(), [&](int i) -> double {
      DLevel& t = built[(size_t)i];
      if (t.fd_steps.empty() && !t.fd_small && !t.fd_cluster) {
        build_fd(L, l, h->opt.delta, h->opt.tau, A, t, cand[(size_t)i]);
        if (cand[(size_t)i] == 2 && !t.fd_small) return -1.0;    // does not fit one CTA
        if (cand[(size_t)i] == 3 && !t.fd_cluster) return -1.0;  // does not fit one cluster
      }
      return time_on_stream(h, [&]() { run_fd(h, t); });
    });
    if (verbose) {
      const auto ts = Tuner::instance().last_times();
      std::fprintf(stderr, "mgiga: tune fd level %d (bucket %d): engine %d;", l, key.bucket, cand[(size_t)choice]);
      for (size_t i = 0; i < ts.size(); ++i) std::fprintf(stderr, " %d: %.4f ms", cand[i], ts[i]);
      std::fprintf(stderr, "\n");
    }
    d = built[(size_t)choice];
    if (d.fd_steps.empty() && !d.fd_small && !d.fd_cluster)
      build_fd(L, l, h->opt.delta, h->opt.tau, A, d, cand[(size_t)choice]);
    return;
  }
  build_fd(L, l, h->opt.delta, h->opt.tau, A, d, cand[(size_t)std::min<int>(choice, (int)cand.size() - 1)]);
}

// autotuned row blocking of the FP32 cycle residual of level l: 1, 2 or 4 threads per row group
void tune_residual(mgiga_handle* h, const Level& L, int l, DLevel& d, bool verbose) {
  const TuneKey key{TUNE_RESIDUAL, L.d, L.p, h->opt.precision, tune_bucket(L.nloc)};
  const int gs[3] = {1, 2, 4};
  const int choice = Tuner::instance().choose(key, 3, [&](int i) -> double {
    d.res_g = gs[i];
    return time_on_stream(h, [&]() { cycle_residual(h, l, d.u, d.f, d.r); });
  });
  d.res_g = gs[choice];
  if (verbose) std::fprintf(stderr, "mgiga: tune residual level %d (bucket %d): %d threads per row group\n", l,
                            key.bucket, d.res_g);
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void mgiga_default_options(mgiga_options* o) {
  if (!o) return;
  o->levels = 0;
  o->smoother = MGIGA_SMOOTHER_SCMS;
  o->nu = 1;
  o->mu = 1;
  o->outer = MGIGA_OUTER_PCG;
  o->precision = MGIGA_PREC_FP64;
  o->max_iter = 1000;
  o->tau = 1.0;
  o->delta = 0.12;
  o->hbm_budget = 0;
  o->stream = nullptr;
  o->gs_cluster = 0;
  o->autotune = 0;
  o->matrix_free = 0;
}

double mgiga_source_sinprod(const double* x, void* ctx) {
  const int d = ctx ? *static_cast<const int*>(ctx) : 2;
  double v = d * M_PI * M_PI;
  for (int a = 0; a < d; ++a) v *= std::sin(M_PI * x[a]);
  return v;
}

mgiga_status mgiga_create(const mgiga_problem* problem, const mgiga_options* opts, mgiga_handle** out) {
  if (!out) return MGIGA_EINVAL;
  *out = nullptr;
  mgiga_handle* h = nullptr;
  try {
    h = new mgiga_handle();
  } catch (...) {
    return MGIGA_ENOMEM;
  }
  *out = h;
  return guarded_call(h, [&]() -> mgiga_status {
    import_problem(problem, h->pr);
    if (opts) h->opt = *opts; else mgiga_default_options(&h->opt);
    const mgiga_options& o = h->opt;
    if (o.smoother < 0 || o.smoother > 2 || o.nu < 1 || o.mu < 1 || o.mu > 2 || o.outer < 0 || o.outer > 1 ||
        o.precision < MGIGA_PREC_FP64 || o.precision > MGIGA_PREC_BF16 || o.max_iter < 0 || !(o.tau > 0.0) || !(o.delta > 0.0) || o.levels < 0 ||
        !(o.gs_cluster == 0 || o.gs_cluster == 2 || o.gs_cluster == 4 || o.gs_cluster == 8 || o.gs_cluster == 16) ||
        o.autotune < 0 || o.autotune > 1 || o.matrix_free < 0 || o.matrix_free > 1)
      throw SetupError(MGIGA_EINVAL, "invalid options");
    h->stream = static_cast<cudaStream_t>(o.stream);
    const int lv = o.levels > 0 ? o.levels : auto_levels(h->pr);
    h->levels = lv;
    init_levels(h->pr, lv, h->L);
    // integer set-up of the smoothers (host only): pieces and colours
    h->colours.assign(lv, {});
    h->pieces.assign(lv, {});
    h->piece_of.assign(lv, {});
    h->num_pieces.assign(lv, 0);
    const int sm = h->opt.smoother;
    for (int l = 1; l < lv; ++l) {
      const Level& L = h->L[l];
      if (sm == MGIGA_SMOOTHER_SCMS || sm == MGIGA_SMOOTHER_HYBRID) {
        h->pieces[l] = decompose(h->pr, L);
        h->piece_of[l].assign(L.ndof, -1);
        for (size_t i = 0; i < h->pieces[l].size(); ++i)
          for (int g : h->pieces[l][i].dofs) h->piece_of[l][g] = (int)i;
        h->num_pieces[l] = (int)h->pieces[l].size();
      }
      if (sm == MGIGA_SMOOTHER_GS || sm == MGIGA_SMOOTHER_HYBRID) h->colours[l] = colouring(h->pr, L);
    }
    return MGIGA_OK;
  });
}

mgiga_status mgiga_assemble(mgiga_handle* h) {
  if (!h) return MGIGA_EINVAL;
  if (h->assembled) return fail(h, MGIGA_ESTATE, "already assembled");
  return guarded_call(h, [&]() -> mgiga_status {
    // every level's FP64 band goes to the device: a lower bound of the footprint,
    // known before the (long) host assembly -- refuse at once what cannot fit
    if (h->opt.hbm_budget) {
      const int W = 2 * h->pr.p + 1;
      const double nb = h->pr.d == 2 ? (double)W * W : (double)W * W * W;
      double lower = 0.0;
      for (const Level& L : h->L) lower += (double)L.nloc * nb * sizeof(double);
      if (lower > (double)h->opt.hbm_budget)
        throw SetupError(MGIGA_ENOMEM, "device footprint exceeds hbm_budget (the FP64 operators alone need " +
                                           std::to_string((long long)lower) + " bytes)");
    }
    // MGIGA_VERBOSE: time of each set-up phase on stderr
    const bool verbose = std::getenv("MGIGA_VERBOSE") != nullptr;
    auto t_last = std::chrono::steady_clock::now();
    auto tick = [&](const char* what, int l) {
      if (!verbose) return;
      const auto now = std::chrono::steady_clock::now();
      std::fprintf(stderr, "mgiga: set-up %-10s level %d: %.3f s\n", what, l,
                   std::chrono::duration<double>(now - t_last).count());
      t_last = now;
    };
    const int lv = h->levels;
    // the level operators' bands are assembled on the GPU (stiffness, Galerkin products) unless the
    // degree is beyond the device kernels or MGIGA_HOST_SETUP=1; the SIPG interface terms, the
    // cross-patch blocks of every level and the transfers stay on the host
    const char* host_env = std::getenv("MGIGA_HOST_SETUP");
    const bool gpu_setup = gpu_setup_supported(h->pr) && !(host_env && host_env[0] == '1');
    // 3D: the element stiffness stays on the host (the device kernel measured slower there: cube,
    // 48 intervals, p = 5: 49 s against 38 s on 16 host cores); its Galerkin products run on the GPU
    const char* s3_env = std::getenv("MGIGA_GPU_STIFFNESS_3D");  // the 3D device kernel, for testing
    // (patches of different degrees: the element stiffness on the host, one degree per patch)
    bool uniform = true;
    for (int k = 0; k < h->pr.K; ++k) uniform = uniform && h->pr.deg(k) == h->pr.p;
    const bool gpu_stiffness = gpu_setup && uniform && (h->pr.d == 2 || (s3_env && s3_env[0] == '1'));
    std::vector<std::pair<int64_t, double>> mf_self;  // within-patch SIPG terms for the matrix-free residual
    if (gpu_setup) {
      Level& F = h->L[lv - 1];
      F.record_band_add = h->opt.matrix_free != 0;
      assemble_fine(h->pr, F, h->pr.knots, /*stiffness=*/!gpu_stiffness);
      if (h->opt.matrix_free) mf_self = F.merged_band_add();
      if (!F.band.empty()) std::vector<std::pair<int64_t, double>>().swap(F.band_add);
      apply_dirichlet(F);
      h->T.assign(lv, Transfer{});
      for (int l = lv - 1; l > 0; --l) {
        h->T[l] = build_transfer(h->L[l - 1], h->L[l]);
        galerkin(h->L[l], h->T[l], h->L[l - 1], /*band=*/false);
        apply_dirichlet(h->L[l - 1]);
      }
      tick("interfaces", lv - 1);
    } else {
      h->L[lv - 1].record_band_add = h->opt.matrix_free != 0;
      assemble_finest(h->pr, h->L);
      if (h->opt.matrix_free) mf_self = h->L[lv - 1].merged_band_add();
      std::vector<std::pair<int64_t, double>>().swap(h->L[lv - 1].band_add);
      tick("assembly", lv - 1);
      galerkin_hierarchy(h->L, h->T);
      tick("galerkin", 0);
    }
    // device: work runs on the caller's stream, or on a non-blocking stream
    // of the handle (the legacy default stream cannot be captured into
    // graphs, and a blocking stream under capture in one thread would fail
    // legacy-stream work of another); the _d entry points order an owned
    // stream after the legacy default stream explicitly
    if (!h->stream) {
      CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
      h->own_stream = true;
    }
    if (!h->legacy_done) CK(cudaEventCreateWithFlags(&h->legacy_done, cudaEventDisableTiming));
    {
      const char* env = std::getenv("MGIGA_SIDE_STREAM");  // 0: the pieces after the interiors, one stream
      if (!h->side && !(env && env[0] == '0')) {
        int prio = 0;
        CK(cudaStreamGetPriority(h->stream, &prio));
        CK(cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, prio));
        CK(cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming));
      }
    }
    CK(cudaGetDevice(&h->device));
    h->arena.reset(new Arena());
    Arena& A = *h->arena;
    A.stream = h->stream;
    if (h->opt.precision == MGIGA_PREC_TF32 || h->opt.precision == MGIGA_PREC_BF16) CK(prepare_gemm_umma());
    A.budget = h->opt.hbm_budget;
    h->D.assign(lv, DLevel{});
    std::vector<double*> dband(lv, nullptr);
    if (gpu_setup) {
      // device bands of every level, finest first, then copied to the host for the set-up steps
      // that read them (interface-piece matrices, Gauss-Seidel blocks, FP32 copies)
      for (int l = 0; l < lv; ++l) dband[l] = A.alloc<double>((size_t)h->L[l].nb * h->L[l].nloc);
      if (gpu_stiffness) {
        gpu_assemble_finest(h->pr, h->L[lv - 1], dband[lv - 1], h->stream);
        tick("gpu stiffness", lv - 1);
      } else {
        const Level& F = h->L[lv - 1];
        CK(cudaMemcpyAsync(dband[lv - 1], F.band.data(), F.band.size() * sizeof(double), cudaMemcpyHostToDevice,
                           h->stream));
        tick("host stiffness", lv - 1);
      }
      for (int l = lv - 1; l > 0; --l) gpu_galerkin_band(h->L[l], h->L[l - 1], h->T[l], dband[l], dband[l - 1], h->stream);
      tick("gpu galerkin", 0);
      for (int l = 0; l < lv; ++l) {
        Level& L = h->L[l];
        if (l == lv - 1 && !gpu_stiffness) continue;  // assembled on the host
        L.band.resize((size_t)L.nb * L.nloc);
        CK(cudaMemcpyAsync(L.band.data(), dband[l], L.band.size() * sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream));
      }
      CK(cudaStreamSynchronize(h->stream));
      tick("download", 0);
    }
    const int sm = h->opt.smoother;
    for (int l = 0; l < lv; ++l) {
      const Level& L = h->L[l];
      DLevel& d = h->D[l];
      d.nloc = L.nloc;
      d.ndof = L.ndof;
      d.K = L.K;
      d.arith = h->opt.precision == MGIGA_PREC_FP64 ? 0 : h->opt.precision == MGIGA_PREC_FP32 ? 1
              : h->opt.precision == MGIGA_PREC_TF32 ? 2 : 3;
      d.guard = guard_of(L);
      d.u = A.guarded(L.nloc, d.guard);
      d.f = A.guarded(L.nloc, d.guard);
      d.r = A.guarded(L.nloc, d.guard);
      d.band = gpu_setup ? dband[l] : A.upload(L.band);
      const bool mf_here = h->opt.matrix_free && l == lv - 1;
      if (mf_here) {
        build_mf(h->pr, L, mf_self, A, d);
        std::vector<std::pair<int64_t, double>>().swap(mf_self);
      }
      if (d.arith >= 1 && l > 0 && !mf_here) {  // FP32 copy for the residuals inside the mixed-precision cycle
        std::vector<float> b32(L.band.size() + 4, 0.0f);
        for (size_t i = 0; i < L.band.size(); ++i) b32[i] = (float)L.band[i];
        d.band32 = A.upload(b32);
      }
      std::vector<PatchMeta> pm(L.K);
      for (int k = 0; k < L.K; ++k) {
        pm[k].off = L.off[k];
        for (int a = 0; a < 3; ++a) pm[k].N[a] = L.N[k][a];
      }
      d.patches = A.upload(pm);
      const auto tiles = make_tiles(L);
      d.tiles = A.upload(tiles);
      d.ntiles = (int)tiles.size();
      d.nx = (int)L.x_row.size();
      d.x_row = A.upload(L.x_row);
      d.x_ptr = A.upload(L.x_ptr);
      d.x_col = A.upload(L.x_col);
      d.x_val = A.upload(L.x_val);
      d.nsh = (int)L.sh_ptr.size() - 1;
      d.sh_ptr = A.upload(L.sh_ptr);
      d.sh_pos = A.upload(L.sh_pos);
      std::vector<int> shp(L.sh_pos.size());
      for (size_t i = 0; i < L.sh_pos.size(); ++i) shp[i] = L.patch_of[L.sh_pos[i]];
      d.sh_patch = A.upload(shp);
      d.weight = conforming(h) ? A.upload(L.weight) : nullptr;
      d.loc2glob = A.upload(L.loc2glob);
      d.owner = A.upload(L.owner);
      if (l >= 1) build_transfer_tables(h->L[l - 1], L, h->T[l], A, d);
      if (l == 0) {
        Piece all;
        all.kind = 1;
        all.patch = -1;
        for (int g = 0; g < L.ndof; ++g) all.dofs.push_back(g);
        build_pieces({all}, L, A, d, true);
        continue;
      }
      tick("uploads", l);
      if (sm == MGIGA_SMOOTHER_SCMS || sm == MGIGA_SMOOTHER_HYBRID) {
        if (h->opt.autotune) tune_fd(h, L, l, A, d, verbose);
        else build_fd(L, l, h->opt.delta, h->opt.tau, A, d);
        tick("fd", l);
        build_pieces(h->pieces[l], L, A, d, false);
        tick("pieces", l);
      }
      if (sm == MGIGA_SMOOTHER_GS || sm == MGIGA_SMOOTHER_HYBRID) build_gs(h->pr, h->colours[l], L, A, d, h->opt.gs_cluster);
      tick("gs", l);
      if (h->opt.autotune && d.band32) tune_residual(h, L, l, d, verbose);
    }
    const Level& Lf = h->L[lv - 1];
    const int64_t g = guard_of(Lf);
    h->x = A.guarded(Lf.nloc, g);
    h->p = A.guarded(Lf.nloc, g);
    h->q = A.guarded(Lf.nloc, g);
    h->b = A.guarded(Lf.nloc, g);
    h->t = A.guarded(Lf.nloc, g);
    h->scal = A.alloc<double>(S_COUNT);
    CK(cudaMemsetAsync(h->scal, 0, S_COUNT * sizeof(double), h->stream));
    h->partials = A.alloc<double>(red_blocks());
    h->counter = A.alloc<unsigned int>(4);
    CK(cudaMemsetAsync(h->counter, 0, 4 * sizeof(unsigned int), h->stream));
    h->gs_bar = A.alloc<unsigned int>(2);
    h->gs_err = A.alloc<int>(1);
    CK(cudaMemsetAsync(h->gs_bar, 0, 2 * sizeof(unsigned int), h->stream));
    CK(cudaMemsetAsync(h->gs_err, 0, sizeof(int), h->stream));
    int maxdof = 1;
    for (const auto& L : h->L) maxdof = std::max(maxdof, L.ndof);
    h->in1 = A.alloc<double>(maxdof);
    h->in2 = A.alloc<double>(maxdof);
    h->out = A.alloc<double>(maxdof);
    CK(cudaMallocHost(&h->host_scal, S_COUNT * sizeof(double)));
    CK(cudaStreamSynchronize(h->stream));
    // the device holds the operators now: keep the nonzero counts, release the host bands
    // (a resident handle otherwise keeps twice its operators' size in host memory)
    for (Level& L : h->L) {
      double nnz = 0.0;
      for (double v : L.band) nnz += v != 0.0;
      L.nnz = nnz;
      Vec().swap(L.band);
    }
    h->assembled = true;
    return MGIGA_OK;
  });
}

mgiga_status mgiga_load(mgiga_handle* h, double (*f)(const double*, void*), void* ctx, double* rhs_out) {
  if (!h || !f || !rhs_out) return h ? fail(h, MGIGA_EINVAL, "NULL argument") : MGIGA_EINVAL;
  return guarded_call(h, [&]() -> mgiga_status {
    assemble_load(h->pr, h->L[h->levels - 1], f, ctx, rhs_out);
    return MGIGA_OK;
  });
}

static mgiga_status apply_impl(mgiga_handle* h, int op, int level, const double* a, const double* b, double* out) {
  if (!h) return MGIGA_EINVAL;
  if (!h->assembled) return fail(h, MGIGA_ESTATE, "mgiga_assemble has not run");
  if (level < 0 || level >= h->levels) return fail(h, MGIGA_EINVAL, "bad level");
  const bool needs_b = op == MGIGA_OP_RESIDUAL || op == MGIGA_OP_SMOOTH || op == MGIGA_OP_GS_FWD ||
                       op == MGIGA_OP_GS_BWD;
  if (!a || !out || (needs_b && !b)) return fail(h, MGIGA_EINVAL, "NULL vector");
  return guarded_call(h, [&]() -> mgiga_status {
    LaunchScope scope(h);
    DLevel& d = h->D[level];
    cudaStream_t st = h->stream;
    const int sm = h->opt.smoother;
    switch (op) {
      case MGIGA_OP_RESIDUAL:
        launch_scatter(d.nloc, st, d.loc2glob, a, d.f);
        launch_scatter(d.nloc, st, d.loc2glob, b, d.u);
        residual(h, level, d.u, d.f, d.r);
        launch_gather(d.ndof, st, d.owner, d.r, out);
        break;
      case MGIGA_OP_CYCLE_RESIDUAL:
        if (level == 0) throw SetupError(MGIGA_EINVAL, "the cycle computes residuals on levels >= 1");
        launch_scatter(d.nloc, st, d.loc2glob, a, d.f);
        launch_scatter(d.nloc, st, d.loc2glob, b, d.u);
        cycle_residual(h, level, d.u, d.f, d.r);
        launch_gather(d.ndof, st, d.owner, d.r, out);
        break;
      case MGIGA_OP_MATVEC:
        launch_scatter(d.nloc, st, d.loc2glob, a, d.u);
        matvec(h, level, d.u, d.r);
        launch_gather(d.ndof, st, d.owner, d.r, out);
        break;
      case MGIGA_OP_SMOOTH:
        if (level == 0 || !(sm == MGIGA_SMOOTHER_SCMS || sm == MGIGA_SMOOTHER_HYBRID))
          throw SetupError(MGIGA_EINVAL, "no subspace-corrected mass smoother on this level");
        launch_scatter(d.nloc, st, d.loc2glob, a, d.f);
        launch_scatter(d.nloc, st, d.loc2glob, b, d.u);
        residual(h, level, d.u, d.f, d.r);
        smooth(h, level);
        launch_gather(d.ndof, st, d.owner, d.u, out);
        break;
      case MGIGA_OP_GS_FWD:
      case MGIGA_OP_GS_BWD:
        if (level == 0 || !(sm == MGIGA_SMOOTHER_GS || sm == MGIGA_SMOOTHER_HYBRID))
          throw SetupError(MGIGA_EINVAL, "no Gauss-Seidel smoother on this level");
        launch_scatter(d.nloc, st, d.loc2glob, a, d.f);
        launch_scatter(d.nloc, st, d.loc2glob, b, d.u);
        gs_sweep(h, level, op == MGIGA_OP_GS_FWD);
        launch_gather(d.ndof, st, d.owner, d.u, out);
        break;
      case MGIGA_OP_RESTRICT:
        if (level == 0) throw SetupError(MGIGA_EINVAL, "restriction needs level >= 1");
        launch_scatter(d.nloc, st, d.loc2glob, a, d.r);
        restrict_to(h, level, d.r);
        launch_gather(h->D[level - 1].ndof, st, h->D[level - 1].owner, h->D[level - 1].f, out);
        break;
      case MGIGA_OP_PROLONG: {
        if (level == 0) throw SetupError(MGIGA_EINVAL, "prolongation needs level >= 1");
        DLevel& c = h->D[level - 1];
        launch_scatter(c.nloc, st, c.loc2glob, a, c.u);
        CK(cudaMemsetAsync(d.u, 0, d.nloc * sizeof(double), st));
        prolong_from(h, level, c.u, d.u);
        launch_gather(d.ndof, st, d.owner, d.u, out);
        break;
      }
      case MGIGA_OP_COARSE:
        if (level != 0) throw SetupError(MGIGA_EINVAL, "the coarse solve lives on level 0");
        launch_scatter(d.nloc, st, d.loc2glob, a, d.f);
        coarse_solve(h);
        launch_gather(d.ndof, st, d.owner, d.u, out);
        break;
      default:
        throw SetupError(MGIGA_EINVAL, "unknown op");
    }
    check_launch();
    CK(cudaStreamSynchronize(st));
    check_device_timeout(h);
    return MGIGA_OK;
  });
}

mgiga_status mgiga_apply_d(mgiga_handle* h, int op, int level, const double* a, const double* b, double* out) {
  if (h && h->assembled) {
    const mgiga_status s = guarded_call(h, [&]() -> mgiga_status {
      after_legacy(h);
      return MGIGA_OK;
    });
    if (s != MGIGA_OK) return s;
  }
  return apply_impl(h, op, level, a, b, out);
}

// ---------------------------------------------------------------------------
// allocation-free residual: its scratch is this fixed device array
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_noalloc_scratch[MGIGA_NOALLOC_SCRATCH_DOUBLES];
static std::mutex g_noalloc_mutex;
static double* g_noalloc_ptr[256] = {nullptr};

// device address of the scratch array on device `dev` (current), looked up once
// per device (the host-side name of the array is not a device address)
static double* noalloc_scratch(int dev) {
  if (dev < 0 || dev >= 256) throw CudaError("device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  return g_noalloc_ptr[dev];
}

mgiga_status mgiga_residual_noalloc_d(mgiga_handle* h, int level, const double* f, const double* u,
                                      double* out) {
  if (!h) return MGIGA_EINVAL;
  if (!h->assembled) return fail(h, MGIGA_ESTATE, "mgiga_assemble has not run");
  if (level < 0 || level >= h->levels) return fail(h, MGIGA_EINVAL, "bad level");
  if (!f || !u || !out) return fail(h, MGIGA_EINVAL, "NULL vector");
  return guarded_call(h, [&]() -> mgiga_status {
    // the scratch of the device that holds the handle's buffers: the call runs there only
    int cur = -1;
    CK(cudaGetDevice(&cur));
    if (cur != h->device)
      return fail(h, MGIGA_EINVAL,
                  "current device " + std::to_string(cur) + " is not the handle's device " + std::to_string(h->device));
    after_legacy(h);
    LaunchScope scope(h);
    const Level& L = h->L[level];
    DLevel& d = h->D[level];
    cudaStream_t st = h->stream;
    // layout: [guard | u | guard] [f] [r], each part 256-byte aligned
    auto up = [](int64_t n) { return (n + 31) / 32 * 32; };
    const int64_t g = up(d.guard), n = up(d.nloc);
    const int64_t need = g + n + g + n + n;
    if (need > (int64_t)MGIGA_NOALLOC_SCRATCH_DOUBLES)
      return fail(h, MGIGA_EINVAL,
                  "level too large for the allocation-free residual: it needs " + std::to_string(need) +
                      " doubles of scratch, the fixed scratch holds " +
                      std::to_string((long long)MGIGA_NOALLOC_SCRATCH_DOUBLES));
    double* base = noalloc_scratch(h->device);
    double* su = base + g;
    double* sf = base + g + n + g;
    double* sr = sf + n;
    // the guards around u must read as zero; the rest is overwritten below
    CK(cudaMemsetAsync(base, 0, (size_t)g * sizeof(double), st));
    CK(cudaMemsetAsync(su + d.nloc, 0, (size_t)(n - d.nloc + g) * sizeof(double), st));
    launch_scatter(d.nloc, st, d.loc2glob, f, sf);
    launch_scatter(d.nloc, st, d.loc2glob, u, su);
    launch_band(L.d, L.p, 0, d.ntiles, st, d.tiles, d.patches, d.band, d.nloc, su, sf, sr);
    launch_cross(0, d.nx, st, d.x_row, d.x_ptr, d.x_col, d.x_val, su, sr);
    if (conforming(h)) launch_shared(d.nsh, st, d.sh_ptr, d.sh_pos, sr, sf, 0);
    launch_gather(d.ndof, st, d.owner, sr, out);
    check_launch();
    CK(cudaStreamSynchronize(st));
    return MGIGA_OK;
  });
}

mgiga_status mgiga_apply(mgiga_handle* h, int op, int level, const double* a, const double* b, double* out) {
  if (!h) return MGIGA_EINVAL;
  if (!h->assembled) return fail(h, MGIGA_ESTATE, "mgiga_assemble has not run");
  if (level < 0 || level >= h->levels) return fail(h, MGIGA_EINVAL, "bad level");
  if (!a || !out) return fail(h, MGIGA_EINVAL, "NULL vector");
  return guarded_call(h, [&]() -> mgiga_status {
    const int nin = (op == MGIGA_OP_PROLONG) ? h->L[level - (level > 0 ? 1 : 0)].ndof : h->L[level].ndof;
    const int nout = (op == MGIGA_OP_RESTRICT) ? h->L[level - (level > 0 ? 1 : 0)].ndof : h->L[level].ndof;
    if (a) CK(cudaMemcpyAsync(h->in1, a, (size_t)nin * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (b) CK(cudaMemcpyAsync(h->in2, b, (size_t)h->L[level].ndof * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    const mgiga_status s = apply_impl(h, op, level, a ? h->in1 : nullptr, b ? h->in2 : nullptr, h->out);
    if (s != MGIGA_OK) return s;
    CK(cudaMemcpyAsync(out, h->out, (size_t)nout * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MGIGA_OK;
  });
}

static void run_vcycle_top(mgiga_handle* h) { vcycle(h, h->levels - 1); }

mgiga_status mgiga_vcycle_d(mgiga_handle* h, const double* r, double* z) {
  if (!h) return MGIGA_EINVAL;
  if (!h->assembled) return fail(h, MGIGA_ESTATE, "mgiga_assemble has not run");
  if (!r || !z) return fail(h, MGIGA_EINVAL, "NULL vector");
  return guarded_call(h, [&]() -> mgiga_status {
    after_legacy(h);
    LaunchScope scope(h);
    DLevel& d = h->D[h->levels - 1];
    launch_scatter(d.nloc, h->stream, d.loc2glob, r, d.f);
    run_vcycle_top(h);
    launch_gather(d.ndof, h->stream, d.owner, d.u, z);
    check_launch();
    CK(cudaStreamSynchronize(h->stream));
    check_device_timeout(h);
    return MGIGA_OK;
  });
}

mgiga_status mgiga_vcycle(mgiga_handle* h, const double* r, double* z) {
  if (!h) return MGIGA_EINVAL;
  if (!h->assembled) return fail(h, MGIGA_ESTATE, "mgiga_assemble has not run");
  if (!r || !z) return fail(h, MGIGA_EINVAL, "NULL vector");
  return guarded_call(h, [&]() -> mgiga_status {
    const int n = h->L[h->levels - 1].ndof;
    CK(cudaMemcpyAsync(h->in1, r, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    const mgiga_status s = mgiga_vcycle_d(h, h->in1, h->out);
    if (s != MGIGA_OK) return s;
    CK(cudaMemcpyAsync(z, h->out, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MGIGA_OK;
  });
}

// A whole PCG solve (Sec. 4) as one graph with conditional nodes (CUDA 12.4+), reading the right-hand
// side and the initial guess from the staging vectors in1 / in2 (global order) and leaving the
// solution in in2:
//   [scatter f, u; ||f||^2; r = f - A u; ||r||^2; cg_ctl_0]
//   if (zero): [u = 0]                      (zero right-hand side)
//   if (go):   [z = B r; (r, z); p = z]     (the first cycle)
//   while (loop): [q = A p, alpha, x += alpha p, r -= alpha q, ||r||^2, cg_ctl_a]
//                 if (confirm): [t = f - A x, ||t||^2, cg_ctl_c]   (the true residual)
//                 if (cont):    [z = B r, beta, p = z + beta p]
//   [gather u]
// so that a solve makes no host round trip until its result.  Returns false (no error left pending)
// when the runtime or the driver cannot build or instantiate it; the host-driven loop is used then.
static void add_if(cudaGraph_t g, const cudaGraphNode_t* dep, cudaGraphConditionalHandle hc, cudaGraphNode_t* node,
                   cudaGraph_t* body, cudaGraphConditionalNodeType type = cudaGraphCondTypeIf) {
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hc;
  cp.conditional.type = type;
  cp.conditional.size = 1;
  CK(cudaGraphAddNode(node, g, dep, nullptr, dep ? 1 : 0, &cp));
  *body = cp.conditional.phGraph_out[0];
}

// the leaf of a graph captured from one stream (a chain)
static cudaGraphNode_t chain_leaf(cudaGraph_t g) {
  size_t nn = 0;
  CK(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  CK(cudaGraphGetNodes(g, nodes.data(), &nn));
  cudaGraphNode_t last = nullptr;
  for (cudaGraphNode_t x : nodes) {
    size_t nd = 0;
    CK(cudaGraphNodeGetDependentNodes(x, nullptr, nullptr, &nd));
    if (nd == 0) last = x;
  }
  return last;
}

static bool build_solve_graph(mgiga_handle* h) {
  const int top = h->levels - 1;
  DLevel& d = h->D[top];
  cudaStream_t st = h->stream;
  const double* w = d.weight;
  const int64_t n = d.nloc;
  double* r = d.f;
  double* z = d.u;
  cudaGraph_t G = nullptr;
  bool ok = false;
  const long long c0 = launch_counter();
  const auto mode = cudaStreamCaptureModeThreadLocal;
  try {
    CK(cudaGraphCreate(&G, 0));
    cudaGraphConditionalHandle hzero, hgo, hloop, hconf, hcont;
    CK(cudaGraphConditionalHandleCreate(&hzero, G, 0, cudaGraphCondAssignDefault));
    CK(cudaGraphConditionalHandleCreate(&hgo, G, 0, cudaGraphCondAssignDefault));
    CK(cudaGraphConditionalHandleCreate(&hloop, G, 0, cudaGraphCondAssignDefault));
    // the start: initial residual and the decision
    CK(cudaStreamBeginCaptureToGraph(st, G, nullptr, nullptr, 0, mode));
    launch_scatter(n, st, d.loc2glob, h->in1, h->b);
    launch_scatter(n, st, d.loc2glob, h->in2, h->x);
    launch_dot(n, st, h->b, h->b, w, h->partials, h->scal, h->counter, S_FF, 0);
    residual(h, top, h->x, h->b, r);
    launch_dot(n, st, r, r, w, h->partials, h->scal, h->counter, S_RR, 0);
    launch_cg_ctl_0(st, h->scal, h->loop_state, h->dhist, hzero, hgo, hloop);
    CK(cudaStreamEndCapture(st, &G));
    const long long k_start = launch_counter() - c0;
    cudaGraphNode_t n0 = chain_leaf(G), nz, ng, nw;
    cudaGraph_t Z, Go, B;
    add_if(G, &n0, hzero, &nz, &Z);
    CK(cudaStreamBeginCaptureToGraph(st, Z, nullptr, nullptr, 0, mode));
    CK(cudaMemsetAsync(h->x, 0, n * sizeof(double), st));
    CK(cudaStreamEndCapture(st, &Z));
    add_if(G, &nz, hgo, &ng, &Go);
    long long c1 = launch_counter();
    CK(cudaStreamBeginCaptureToGraph(st, Go, nullptr, nullptr, 0, mode));
    vcycle(h, top);
    launch_dot(n, st, r, z, w, h->partials, h->scal, h->counter, S_RZ, 0);
    CK(cudaMemcpyAsync(h->p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamEndCapture(st, &Go));
    const long long k_go = launch_counter() - c1;
    add_if(G, &ng, hloop, &nw, &B, cudaGraphCondTypeWhile);
    CK(cudaGraphConditionalHandleCreate(&hconf, B, 0, 0));
    CK(cudaGraphConditionalHandleCreate(&hcont, B, 0, 0));
    // loop body: first half of an iteration
    CK(cudaStreamBeginCaptureToGraph(st, B, nullptr, nullptr, 0, mode));
    matvec(h, top, h->p, h->q);
    launch_dot(n, st, h->p, h->q, w, h->partials, h->scal, h->counter, S_PQ, 1);
    launch_cg_xr(n, st, h->x, r, h->p, h->q, w, h->partials, h->scal, h->counter);
    launch_cg_ctl_a(st, h->scal, h->loop_state, h->dhist, hloop, hconf, hcont);
    CK(cudaStreamEndCapture(st, &B));
    cudaGraphNode_t nb0 = chain_leaf(B), nc, nn2;
    cudaGraph_t C, D;
    add_if(B, &nb0, hconf, &nc, &C);
    c1 = launch_counter();
    CK(cudaStreamBeginCaptureToGraph(st, C, nullptr, nullptr, 0, mode));
    residual(h, top, h->x, h->b, h->t);
    launch_dot(n, st, h->t, h->t, w, h->partials, h->scal, h->counter, S_TMP, 0);
    launch_cg_ctl_c(st, h->scal, h->loop_state, h->dhist, hloop, hcont);
    CK(cudaStreamEndCapture(st, &C));
    h->g_conf_kernels = launch_counter() - c1;
    add_if(B, &nc, hcont, &nn2, &D);
    CK(cudaStreamBeginCaptureToGraph(st, D, nullptr, nullptr, 0, mode));
    const bool flexible = h->opt.precision != MGIGA_PREC_FP64;
    if (flexible) launch_dot(n, st, r, z, w, h->partials, h->scal, h->counter, S_RZOLD, 0);
    vcycle(h, top);
    launch_dot(n, st, r, z, w, h->partials, h->scal, h->counter, S_RZNEW, flexible ? 3 : 2);
    launch_cg_p(n, st, h->p, z, h->scal);
    CK(cudaStreamEndCapture(st, &D));
    // the end: the solution into in2
    CK(cudaStreamBeginCaptureToGraph(st, G, &nw, nullptr, 1, mode));
    launch_gather(d.ndof, st, d.owner, h->x, h->in2);
    CK(cudaStreamEndCapture(st, &G));
    CK(cudaGraphInstantiate(&h->g_solve, G, 0));
    h->g_start_kernels = k_start + 1;  // + the gather at the end
    h->g_go_kernels = k_go;
    h->g_solve_tmpl = G;
    G = nullptr;
    ok = true;
  } catch (const std::exception&) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(st, &junk);
      if (junk && junk != G) cudaGraphDestroy(junk);
    }
    cudaGetLastError();  // leave no error pending
    if (h->g_solve) { cudaGraphExecDestroy(h->g_solve); h->g_solve = nullptr; }
  }
  if (G) cudaGraphDestroy(G);
  h->launches -= launch_counter() - c0;  // captured, not run
  return ok;
}

// the device-driven loop unless MGIGA_DEVICE_LOOP=0; built on first use (needs the kernel counts of
// the host loop's two graphs for the launch statistics, so those are captured too)
static bool use_device_loop(mgiga_handle* h) {
  if (h->device_loop < 0) return false;
  if (const char* env = std::getenv("MGIGA_DEVICE_LOOP"))
    if (env[0] == '0') return false;
  if (h->device_loop == 0) {
    if (!h->loop_state) {
      h->loop_state = h->arena->alloc<CgLoopState>(1);
      h->dhist = h->arena->alloc<double>((size_t)h->opt.max_iter + 2);
      CK(cudaMallocHost(&h->host_state, sizeof(CgLoopState)));
    }
    const int top = h->levels - 1;
    DLevel& d = h->D[top];
    cudaStream_t st = h->stream;
    const double* w = d.weight;
    const int64_t n = d.nloc;
    // kernel counts of the halves (for mgiga_kernel_launches), from dry captures
    if (!h->g_iter_a_kernels) {
      cudaGraph_t g;
      long long c0 = launch_counter();
      CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      matvec(h, top, h->p, h->q);
      launch_dot(n, st, h->p, h->q, w, h->partials, h->scal, h->counter, S_PQ, 1);
      launch_cg_xr(n, st, h->x, d.f, h->p, h->q, w, h->partials, h->scal, h->counter);
      CK(cudaStreamEndCapture(st, &g));
      cudaGraphDestroy(g);
      h->g_iter_a_kernels = launch_counter() - c0 + 1;  // + the control kernel
      c0 = launch_counter();
      CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      const bool flexible = h->opt.precision != MGIGA_PREC_FP64;
      if (flexible) launch_dot(n, st, d.f, d.u, w, h->partials, h->scal, h->counter, S_RZOLD, 0);
      vcycle(h, top);
      launch_dot(n, st, d.f, d.u, w, h->partials, h->scal, h->counter, S_RZNEW, flexible ? 3 : 2);
      launch_cg_p(n, st, h->p, d.u, h->scal);
      CK(cudaStreamEndCapture(st, &g));
      cudaGraphDestroy(g);
      h->g_iter_b_kernels = launch_counter() - c0;
      h->launches -= h->g_iter_a_kernels - 1 + h->g_iter_b_kernels;
    }
    h->device_loop = build_solve_graph(h) ? 1 : -1;
  }
  return h->device_loop > 0;
}

// PCG (Sec. 4) or the cycle as solver, on device-resident global vectors
// enqueue a whole PCG solve as one graph launch (rhs, u: device vectors in global order; u is
// read as the initial guess and receives the solution); no host synchronisation
static void enqueue_graph_solve(mgiga_handle* h, const double* rhs, double* u, double tol) {
  cudaStream_t st = h->stream;
  const size_t bytes = (size_t)h->L[h->levels - 1].ndof * sizeof(double);
  if (rhs != h->in1) CK(cudaMemcpyAsync(h->in1, rhs, bytes, cudaMemcpyDeviceToDevice, st));
  if (u != h->in2) CK(cudaMemcpyAsync(h->in2, u, bytes, cudaMemcpyDeviceToDevice, st));
  launch_cg_loop_init(st, h->scal, h->loop_state, tol, 0.0, h->opt.max_iter);
  check_launch();
  CK(cudaGraphLaunch(h->g_solve, st));
  if (u != h->in2) CK(cudaMemcpyAsync(u, h->in2, bytes, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(h->host_state, h->loop_state, sizeof(CgLoopState), cudaMemcpyDeviceToHost, st));
  h->pending = true;
}

// after the stream of an enqueued graph solve has drained: status, iterations, history
static mgiga_status finish_graph_solve(mgiga_handle* h, int* iters, double* final_relres) {
  h->pending = false;
  const CgLoopState ls = *h->host_state;
  const int it = ls.it;
  if (iters) *iters = it;
  if (final_relres) *final_relres = ls.rel;
  h->history.clear();
  h->launches += h->g_start_kernels;
  if (ls.status == 4) return fail(h, MGIGA_EBREAKDOWN, "non-finite right-hand side or initial guess");
  if (it > 0) h->launches += h->g_go_kernels;  // the first cycle ran iff the loop did
  h->launches += (long long)it * h->g_iter_a_kernels + (long long)ls.nconf * h->g_conf_kernels +
                 (long long)ls.ncont * h->g_iter_b_kernels;
  std::vector<double> hh((size_t)it + 1);
  CK(cudaMemcpy(hh.data(), h->dhist, hh.size() * sizeof(double), cudaMemcpyDeviceToHost));
  h->history = hh;
  check_device_timeout(h);
  if (ls.status == 3) return fail(h, MGIGA_EBREAKDOWN, "CG breakdown (p^T A p <= 0 or NaN)");
  if (ls.status == 2) return fail(h, MGIGA_ENOCONV, "max_iter reached");
  return MGIGA_OK;
}

static mgiga_status solve_impl(mgiga_handle* h, const double* rhs, double* u, double tol, int* iters,
                               double* final_relres) {
  h->history.clear();  // a solve that fails early leaves its own (empty or partial) history
  if (h->opt.outer == MGIGA_OUTER_PCG && use_device_loop(h)) {
    {
      LaunchScope scope(h);
      enqueue_graph_solve(h, rhs, u, tol);
    }
    CK(cudaStreamSynchronize(h->stream));
    return finish_graph_solve(h, iters, final_relres);
  }
  LaunchScope scope(h);
  const int top = h->levels - 1;
  DLevel& d = h->D[top];
  cudaStream_t st = h->stream;
  const double* w = d.weight;
  const int64_t n = d.nloc;
  double* r = d.f;  // CG residual = input of the cycle
  double* z = d.u;  // cycle output
  auto read_scal = [&]() {
    CK(cudaMemcpyAsync(h->host_scal, h->scal, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  };
  launch_scatter(n, st, d.loc2glob, rhs, h->b);
  launch_scatter(n, st, d.loc2glob, u, h->x);
  launch_dot(n, st, h->b, h->b, w, h->partials, h->scal, h->counter, S_FF, 0);
  residual(h, top, h->x, h->b, r);
  launch_dot(n, st, r, r, w, h->partials, h->scal, h->counter, S_RR, 0);
  check_launch();
  read_scal();
  const double ff = h->host_scal[S_FF];
  if (iters) *iters = 0;
  if (!std::isfinite(ff) || !std::isfinite(h->host_scal[S_RR]))
    return fail(h, MGIGA_EBREAKDOWN, "non-finite right-hand side or initial guess");
  if (!(ff > 0.0)) {
    // zero right-hand side: the solution is zero
    CK(cudaMemsetAsync(h->x, 0, n * sizeof(double), st));
    launch_gather(d.ndof, st, d.owner, h->x, u);
    CK(cudaStreamSynchronize(st));
    if (final_relres) *final_relres = 0.0;
    h->history.push_back(0.0);
    return MGIGA_OK;
  }
  const double nf = std::sqrt(ff);
  double rel = std::sqrt(h->host_scal[S_RR]) / nf;
  h->history.push_back(rel);
  const int maxit = h->opt.max_iter;
  int it = 0;
  bool converged = rel <= tol;
  if (h->opt.outer == MGIGA_OUTER_DIRECT) {
    // u <- MG(L, f, u): the cycle on the error equation, u += B (f - A u)
    while (!converged && it < maxit) {
      vcycle(h, top);
      launch_axpby((int64_t)n, st, 1.0, z, 1.0, h->x);
      residual(h, top, h->x, h->b, r);
      launch_dot(n, st, r, r, w, h->partials, h->scal, h->counter, S_RR, 0);
      check_launch();
      read_scal();
      ++it;
      rel = std::sqrt(h->host_scal[S_RR]) / nf;
      h->history.push_back(rel);
      if (!std::isfinite(rel)) return fail(h, MGIGA_EBREAKDOWN, "non-finite residual");
      converged = rel <= tol;
    }
  } else if (!converged) {
    // capture the two halves of a PCG iteration once per handle
    if (!h->g_iter_a) {
      cudaGraph_t g;
      long long c0 = launch_counter();
      CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      matvec(h, top, h->p, h->q);
      launch_dot(n, st, h->p, h->q, w, h->partials, h->scal, h->counter, S_PQ, 1);
      launch_cg_xr(n, st, h->x, r, h->p, h->q, w, h->partials, h->scal, h->counter);
      CK(cudaStreamEndCapture(st, &g));
      CK(cudaGraphInstantiate(&h->g_iter_a, g, 0));
      cudaGraphDestroy(g);
      h->g_iter_a_kernels = launch_counter() - c0;
      c0 = launch_counter();
      CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      // the mixed-precision cycle is not exactly a fixed symmetric operator:
      // flexible (Polak-Ribiere) beta, which needs r_new . z_old
      const bool flexible = h->opt.precision != MGIGA_PREC_FP64;
      if (flexible) launch_dot(n, st, r, z, w, h->partials, h->scal, h->counter, S_RZOLD, 0);
      vcycle(h, top);
      launch_dot(n, st, r, z, w, h->partials, h->scal, h->counter, S_RZNEW, flexible ? 3 : 2);
      launch_cg_p(n, st, h->p, z, h->scal);
      CK(cudaStreamEndCapture(st, &g));
      CK(cudaGraphInstantiate(&h->g_iter_b, g, 0));
      cudaGraphDestroy(g);
      h->g_iter_b_kernels = launch_counter() - c0;
      // captured kernels did not run: only graph launches count
      h->launches -= h->g_iter_a_kernels + h->g_iter_b_kernels;
    }
    vcycle(h, top);
    launch_dot(n, st, r, z, w, h->partials, h->scal, h->counter, S_RZ, 0);
    CK(cudaMemcpyAsync(h->p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    check_launch();
    while (it < maxit) {
      CK(cudaGraphLaunch(h->g_iter_a, st));
      h->launches += h->g_iter_a_kernels;
      read_scal();
      ++it;
      const double pq = h->host_scal[S_PQ];
      rel = std::sqrt(h->host_scal[S_RR]) / nf;
      h->history.push_back(rel);
      if (!(pq > 0.0) || !std::isfinite(rel)) return fail(h, MGIGA_EBREAKDOWN, "CG breakdown (p^T A p <= 0 or NaN)");
      if (rel <= tol) {
        // confirm with the true residual
        residual(h, top, h->x, h->b, h->t);
        launch_dot(n, st, h->t, h->t, w, h->partials, h->scal, h->counter, S_TMP, 0);
        check_launch();
        read_scal();
        const double trel = std::sqrt(h->host_scal[S_TMP]) / nf;
        if (trel <= tol) {  // the history ends with the confirmed (true) residual
          rel = trel;
          h->history.back() = trel;
          converged = true;
          break;
        }
      }
      if (it >= maxit) break;
      CK(cudaGraphLaunch(h->g_iter_b, st));
      h->launches += h->g_iter_b_kernels;
    }
  }
  launch_gather(d.ndof, st, d.owner, h->x, u);
  check_launch();
  CK(cudaStreamSynchronize(st));
  check_device_timeout(h);
  if (iters) *iters = it;
  if (final_relres) *final_relres = rel;
  return converged ? MGIGA_OK : fail(h, MGIGA_ENOCONV, "max_iter reached");
}

mgiga_status mgiga_solve_d(mgiga_handle* h, const double* rhs, double* u, double tol, int* iters,
                           double* final_relres) {
  if (!h) return MGIGA_EINVAL;
  if (!h->assembled) return fail(h, MGIGA_ESTATE, "mgiga_assemble has not run");
  if (!rhs || !u) return fail(h, MGIGA_EINVAL, "NULL vector");
  return guarded_call(h, [&]() {
    after_legacy(h);
    return solve_impl(h, rhs, u, tol, iters, final_relres);
  });
}

mgiga_status mgiga_solve(mgiga_handle* h, const double* rhs, double* u, double tol, int* iters,
                         double* final_relres) {
  if (!h) return MGIGA_EINVAL;
  if (!h->assembled) return fail(h, MGIGA_ESTATE, "mgiga_assemble has not run");
  if (!rhs || !u) return fail(h, MGIGA_EINVAL, "NULL vector");
  return guarded_call(h, [&]() -> mgiga_status {
    const int n = h->L[h->levels - 1].ndof;
    CK(cudaMemcpyAsync(h->in1, rhs, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->in2, u, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    const mgiga_status s = solve_impl(h, h->in1, h->in2, tol, iters, final_relres);
    if (s == MGIGA_OK || s == MGIGA_ENOCONV) {
      CK(cudaMemcpyAsync(u, h->in2, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
    }
    return s;
  });
}

// ---------------------------------------------------------------------------
// batched solves: many handles, one host pass
// ---------------------------------------------------------------------------
namespace {
// one graph for a whole batch: per problem the staging copies, the parameters, the problem's solve graph
// (a child graph) and the copies back, all problems' chains side by side; rebuilt when the batch changes
struct BatchGraph {
  std::vector<mgiga_handle*> hs;
  std::vector<const double*> rhs;
  std::vector<double*> u;
  std::vector<double> tol;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t stream = nullptr;
  ~BatchGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (stream) cudaStreamDestroy(stream);
  }
};
std::mutex g_batch_mutex;
std::unique_ptr<BatchGraph> g_batch;

bool build_batch_graph(BatchGraph& bg) {
  cudaGraph_t G = nullptr;
  bool ok = false;
  try {
    CK(cudaGraphCreate(&G, 0));
    for (size_t i = 0; i < bg.hs.size(); ++i) {
      mgiga_handle* h = bg.hs[i];
      const size_t bytes = (size_t)h->L[h->levels - 1].ndof * sizeof(double);
      cudaGraphNode_t a, b, c, k, e, f;
      CK(cudaGraphAddMemcpyNode1D(&a, G, nullptr, 0, h->in1, bg.rhs[i], bytes, cudaMemcpyDeviceToDevice));
      CK(cudaGraphAddMemcpyNode1D(&b, G, &a, 1, h->in2, bg.u[i], bytes, cudaMemcpyDeviceToDevice));
      // the parameters of the solve: a captured launch of the init kernel
      cudaGraph_t init = nullptr;
      cudaStream_t cs = h->stream;
      CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      launch_cg_loop_init(cs, h->scal, h->loop_state, bg.tol[i], 0.0, h->opt.max_iter);
      CK(cudaStreamEndCapture(cs, &init));
      const cudaError_t e1 = cudaGraphAddChildGraphNode(&c, G, &b, 1, init);
      cudaGraphDestroy(init);
      CK(e1);
      CK(cudaGraphAddChildGraphNode(&k, G, &c, 1, h->g_solve_tmpl));
      CK(cudaGraphAddMemcpyNode1D(&e, G, &k, 1, bg.u[i], h->in2, bytes, cudaMemcpyDeviceToDevice));
      CK(cudaGraphAddMemcpyNode1D(&f, G, &e, 1, h->host_state, h->loop_state, sizeof(CgLoopState),
                                  cudaMemcpyDeviceToHost));
    }
    CK(cudaGraphInstantiate(&bg.exec, G, 0));
    ok = true;
  } catch (const std::exception&) {
    cudaGetLastError();
    if (bg.exec) { cudaGraphExecDestroy(bg.exec); bg.exec = nullptr; }
  }
  if (G) cudaGraphDestroy(G);
  return ok;
}
}  // namespace

mgiga_status mgiga_solve_batch_d(mgiga_handle* const* hs, int n, const double* const* rhs, double* const* u,
                                 double tol, int flags, int* iters, double* final_relres, int* status) {
  if (n < 0 || (n > 0 && (!hs || !rhs || !u))) return MGIGA_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return MGIGA_EINVAL;
    if (!hs[i]->assembled) return fail(hs[i], MGIGA_ESTATE, "mgiga_assemble has not run");
    if (!rhs[i] || !u[i]) return fail(hs[i], MGIGA_EINVAL, "NULL vector");
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(hs[i], MGIGA_EINVAL, "a handle appears twice in the batch");
  }
  std::vector<int> st(n, MGIGA_OK), graph(n, 0);
  // every solve enqueued before any is awaited
  for (int i = 0; i < n; ++i) {
    mgiga_handle* h = hs[i];
    st[i] = guarded_call(h, [&]() -> mgiga_status {
      after_legacy(h);
      h->history.clear();
      if (h->opt.outer != MGIGA_OUTER_PCG || !use_device_loop(h)) return MGIGA_OK;  // solved below, alone
      graph[i] = 1;
      return MGIGA_OK;
    });
  }
  bool one_graph = false;
  if ((flags & MGIGA_BATCH_ONE_GRAPH) && n > 0) {
    bool all = true;
    for (int i = 0; i < n; ++i) all = all && graph[i] && st[i] == MGIGA_OK && hs[i]->g_solve_tmpl;
    if (all) {
      std::lock_guard<std::mutex> lock(g_batch_mutex);
      const bool same = g_batch && g_batch->hs == std::vector<mgiga_handle*>(hs, hs + n) &&
                        g_batch->rhs == std::vector<const double*>(rhs, rhs + n) &&
                        g_batch->u == std::vector<double*>(u, u + n) && g_batch->tol == std::vector<double>(n, tol);
      if (!same) {
        std::unique_ptr<BatchGraph> bg(new BatchGraph());
        bg->hs.assign(hs, hs + n);
        bg->rhs.assign(rhs, rhs + n);
        bg->u.assign(u, u + n);
        bg->tol.assign(n, tol);
        if (cudaStreamCreateWithFlags(&bg->stream, cudaStreamNonBlocking) == cudaSuccess && build_batch_graph(*bg))
          g_batch = std::move(bg);
        else
          g_batch.reset();
      }
      if (g_batch && g_batch->exec) {
        // the batch's stream starts after every handle's earlier work
        for (int i = 0; i < n; ++i) {
          cudaEvent_t ev;
          if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
            cudaEventRecord(ev, hs[i]->stream);
            cudaStreamWaitEvent(g_batch->stream, ev, 0);
            cudaEventDestroy(ev);
          }
        }
        if (cudaGraphLaunch(g_batch->exec, g_batch->stream) == cudaSuccess &&
            cudaStreamSynchronize(g_batch->stream) == cudaSuccess) {
          one_graph = true;
          for (int i = 0; i < n; ++i) hs[i]->pending = true;
        }
      }
    }
  }
  if (!one_graph)
    for (int i = 0; i < n; ++i) {
      if (!graph[i] || st[i] != MGIGA_OK) continue;
      mgiga_handle* h = hs[i];
      st[i] = guarded_call(h, [&]() -> mgiga_status {
        LaunchScope scope(h);
        enqueue_graph_solve(h, rhs[i], u[i], tol);
        return MGIGA_OK;
      });
    }
  mgiga_status first = MGIGA_OK;
  for (int i = 0; i < n; ++i) {
    mgiga_handle* h = hs[i];
    int it = 0;
    double rel = 0.0;
    if (st[i] == MGIGA_OK) {
      if (graph[i])
        st[i] = guarded_call(h, [&]() -> mgiga_status {
          CK(cudaStreamSynchronize(h->stream));
          return finish_graph_solve(h, &it, &rel);
        });
      else
        st[i] = guarded_call(h, [&]() { return solve_impl(h, rhs[i], u[i], tol, &it, &rel); });
    }
    if (iters) iters[i] = it;
    if (final_relres) final_relres[i] = rel;
    if (status) status[i] = st[i];
    if (first == MGIGA_OK && st[i] != MGIGA_OK) first = (mgiga_status)st[i];
  }
  return first;
}

mgiga_status mgiga_check_wait_expiry(mgiga_handle* h, long long iterations, double* elapsed_ms) {
  if (!h) return MGIGA_EINVAL;
  if (!h->assembled) return fail(h, MGIGA_ESTATE, "mgiga_assemble has not run");
  if (iterations < 1 || iterations > kMbarPolls) return fail(h, MGIGA_EINVAL, "iterations outside [1, 2^18]");
  return guarded_call(h, [&]() -> mgiga_status {
    if (!h->probe_ns) h->probe_ns = h->arena->alloc<long long>(1);
    {
      LaunchScope scope(h);
      launch_wait_expiry_probe(iterations, h->stream, h->gs_err, h->probe_ns);
      check_launch();
    }
    long long ns = 0;
    CK(cudaMemcpyAsync(&ns, h->probe_ns, sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (elapsed_ms) *elapsed_ms = ns * 1e-6;
    check_device_timeout(h);
    return MGIGA_OK;
  });
}

mgiga_status mgiga_residual_history(const mgiga_handle* h, double* out, int cap, int* n) {
  if (!h || !n || cap < 0 || (cap > 0 && !out)) return MGIGA_EINVAL;
  *n = (int)h->history.size();
  for (int i = 0; i < std::min(cap, *n); ++i) out[i] = h->history[(size_t)i];
  return MGIGA_OK;
}

mgiga_status mgiga_kernel_launches(const mgiga_handle* h, long long* n) {
  if (!h || !n) return MGIGA_EINVAL;
  *n = h->launches;
  return MGIGA_OK;
}

static void run_stage(mgiga_handle* h, int stage, int level) {
  const Level& L = h->L[level];
  DLevel& d = h->D[level];
  switch (stage) {
    case MGIGA_STAGE_BAND:
      launch_band(L.d, L.p, 1, d.ntiles, h->stream, d.tiles, d.patches, d.band, d.nloc, d.u, nullptr, d.r);
      break;
    case MGIGA_STAGE_RESIDUAL:
      cycle_residual(h, level, d.u, d.f, d.r);
      break;
    case MGIGA_STAGE_FD:
      run_fd(h, d);
      break;
    case MGIGA_STAGE_PIECES:
      launch_piece(d.npiece_items, d.piece_max_n, h->stream, d.piece_items, d.pieces, d.zpool, d.zpool_f32, d.piece_pos, d.r,
                   d.u, h->opt.tau, 0);
      break;
    case MGIGA_STAGE_GS: gs_sweep(h, level, true); break;
    case MGIGA_STAGE_RESTRICT: restrict_to(h, level, d.r, true); break;
    case MGIGA_STAGE_PROLONG: prolong_from(h, level, h->D[level - 1].u, d.u, true); break;
    case MGIGA_STAGE_COARSE: coarse_solve(h); break;
    case MGIGA_STAGE_VCYCLE: vcycle(h, level); break;
    default: throw SetupError(MGIGA_EINVAL, "unknown stage");
  }
}

static bool stage_valid(const mgiga_handle* h, int stage, int level) {
  const int sm = h->opt.smoother;
  const bool scms = sm == MGIGA_SMOOTHER_SCMS || sm == MGIGA_SMOOTHER_HYBRID;
  const bool gs = sm == MGIGA_SMOOTHER_GS || sm == MGIGA_SMOOTHER_HYBRID;
  switch (stage) {
    case MGIGA_STAGE_BAND: case MGIGA_STAGE_VCYCLE: return true;
    case MGIGA_STAGE_FD: case MGIGA_STAGE_PIECES: return scms && level >= 1;
    case MGIGA_STAGE_GS: return gs && level >= 1;
    case MGIGA_STAGE_RESTRICT: case MGIGA_STAGE_PROLONG: case MGIGA_STAGE_RESIDUAL: return level >= 1;
    case MGIGA_STAGE_COARSE: return level == 0;
    default: return false;
  }
}

mgiga_status mgiga_time_stage(mgiga_handle* h, int stage, int level, int reps, double* ms) {
  if (!h || !ms || reps < 1) return MGIGA_EINVAL;
  if (!h->assembled) return fail(h, MGIGA_ESTATE, "mgiga_assemble has not run");
  if (level < 0 || level >= h->levels || !stage_valid(h, stage, level)) return fail(h, MGIGA_EINVAL, "bad stage/level");
  return guarded_call(h, [&]() -> mgiga_status {
    LaunchScope scope(h);
    struct Events {  // destroyed on every exit, also when a CUDA error throws
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      ~Events() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
      }
    } ev;
    CK(cudaEventCreate(&ev.e0));
    CK(cudaEventCreate(&ev.e1));
    run_stage(h, stage, level);  // warm-up
    CK(cudaEventRecord(ev.e0, h->stream));
    for (int i = 0; i < reps; ++i) run_stage(h, stage, level);
    CK(cudaEventRecord(ev.e1, h->stream));
    check_launch();
    CK(cudaEventSynchronize(ev.e1));
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, ev.e0, ev.e1));
    check_device_timeout(h);
    *ms = (double)t / reps;
    return MGIGA_OK;
  });
}

mgiga_status mgiga_stage_work(const mgiga_handle* h, int stage, int level, double* flops, double* bytes) {
  if (!h || level < 0 || level >= h->levels) return MGIGA_EINVAL;
  if (!stage_valid(h, stage, level)) return MGIGA_EINVAL;
  const Level& L = h->L[level];
  if (!h->assembled) return MGIGA_ESTATE;  // operators are assembled by mgiga_assemble
  // the mixed path keeps FP32 band copies for the cycle's residuals (levels >= 1) and sweeps
  const bool f32 = h->opt.precision != MGIGA_PREC_FP64;
  double fl = 0.0, by = 0.0;
  if (stage == MGIGA_STAGE_RESIDUAL && h->D[level].mf) {
    // matrix-free: the sum-factorised passes and the pointwise flux (2 flops per FMA); u and f read,
    // out written, the window partials written and read back
    fl = h->D[level].mf_flops;
    by = h->D[level].mf_bytes;
  } else if (stage == MGIGA_STAGE_BAND || stage == MGIGA_STAGE_RESIDUAL) {
    // every nonzero once (FP32 coefficients for the residual of the mixed path), u and f read, out written
    const double nnz = L.nnz;
    fl = 2.0 * nnz;
    by = (stage == MGIGA_STAGE_RESIDUAL && f32 && level > 0 ? 4.0 : 8.0) * nnz + 24.0 * (double)L.nloc;
  } else if (stage == MGIGA_STAGE_FD) {
    for (int k = 0; k < L.K; ++k) {
      double nint = 1.0, sum = 0.0;
      for (int a = 0; a < L.d; ++a) { nint *= L.N[k][a] - 2; sum += L.N[k][a] - 2; }
      fl += 4.0 * sum * nint;  // forward and inverse transform: 2 * 2 n_a per DoF and direction
      by += 24.0 * nint;
    }
  } else if (stage == MGIGA_STAGE_GS) {
    // every nonzero once (FP32 coefficients on the mixed path), u read and written, f read
    const double nnz = L.nnz;
    fl = 2.0 * nnz;
    by = (f32 ? 4.0 : 8.0) * nnz + 24.0 * (double)L.nloc;
  } else {
    return MGIGA_EINVAL;
  }
  if (flops) *flops = fl;
  if (bytes) *bytes = by;
  return MGIGA_OK;
}

mgiga_status mgiga_num_levels(const mgiga_handle* h, int* levels) {
  if (!h || !levels) return MGIGA_EINVAL;
  *levels = h->levels;
  return MGIGA_OK;
}

mgiga_status mgiga_ndof(const mgiga_handle* h, int level, long* n) {
  if (!h || !n || level < 0 || level >= h->levels) return MGIGA_EINVAL;
  *n = h->L[level].ndof;
  return MGIGA_OK;
}

mgiga_status mgiga_dof_map(const mgiga_handle* h, int level, int* patch, int* local_index) {
  if (!h || level < 0 || level >= h->levels) return MGIGA_EINVAL;
  const Level& L = h->L[level];
  for (int g = 0; g < L.ndof; ++g) {
    const int64_t pos = L.owner[g];
    const int k = L.patch_of[pos];
    if (patch) patch[g] = k;
    if (local_index) local_index[g] = (int)(pos - L.off[k]);
  }
  return MGIGA_OK;
}

mgiga_status mgiga_colours(const mgiga_handle* h, int level, int* colour) {
  if (!h || !colour || level < 0 || level >= h->levels) return MGIGA_EINVAL;
  if ((int)h->colours.size() <= level || h->colours[level].empty()) return MGIGA_ESTATE;
  std::copy(h->colours[level].begin(), h->colours[level].end(), colour);
  return MGIGA_OK;
}

mgiga_status mgiga_pieces(const mgiga_handle* h, int level, int* piece_of, int* num_pieces) {
  if (!h || !piece_of || level < 0 || level >= h->levels) return MGIGA_EINVAL;
  if ((int)h->piece_of.size() <= level || h->piece_of[level].empty()) return MGIGA_ESTATE;
  std::copy(h->piece_of[level].begin(), h->piece_of[level].end(), piece_of);
  if (num_pieces) *num_pieces = h->num_pieces[level];
  return MGIGA_OK;
}

mgiga_status mgiga_device_bytes(const mgiga_handle* h, size_t* bytes) {
  if (!h || !bytes) return MGIGA_EINVAL;
  *bytes = h->arena ? h->arena->bytes : 0;
  return MGIGA_OK;
}

const char* mgiga_last_error(const mgiga_handle* h) { return h ? h->err.c_str() : "NULL handle"; }

void mgiga_destroy(mgiga_handle* h) { delete h; }

}  // extern "C"
