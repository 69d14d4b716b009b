// Launchers of the device kernels (kernels.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "device.cuh"

namespace mgiga {
namespace dev {


// arguments of the cooperative Gauss-Seidel sweep (all colours, one launch)
struct GsSweepArgs {
  int c_begin, c_end, forward;  // colours [c_begin, c_end), ascending if forward
  const int* cptr;        // ncol + 1 entry offsets (device)
  int64_t ngs;            // number of entries (= ndof)
  const void* gsband;     // band rows of the owner copies in colour order, gsband[o * ngs + e]
                          // (double, or float for the mixed path)
  const int64_t* gs_pos;  // owner position of entry e
  const int2* gs_stride;  // (N_0, N_0 N_1) of its patch
  const int2* gs_xrange;  // its couplings besides its band row, entries [x, y) of x_col / x_val: the
                          // SIPG couplings, then the band rows of a shared DoF's further copies
  const int* gs_cls;      // shared class (conforming) or -1
  const PatchMeta* patches;
  const double* band;
  int64_t nloc;
  const int* sh_ptr;
  const int64_t* sh_pos;
  const int* sh_patch;
  const int64_t* x_col;
  const double* x_val;
  const double* f;
  double* u;
  unsigned int* bar;  // [count, generation], count 0 at launch
  int* err;           // set to 1 when a barrier wait gives up
};
int gs_coop_max_blocks(int d, int p, bool f32);
cudaError_t launch_gs_sweep(int d, int p, bool f32, int blocks, cudaStream_t st, GsSweepArgs a);
// staged patch-parallel phase of the mixed path (FP32 coefficient blocks)
struct GsStagedArgs {
  int c_begin, c_end, forward;  // base colours of the phase, sweep direction
  int K, csize, base;           // patches, CTAs per patch cluster, base colours per parity
  int nbuf, cap;                // chunk buffers of cap bytes (1: the CTA's whole phase at once; else a ring)
  int threads, tpr;             // CTA size (256, 512 or 1024) and threads per row (4..32, power of two)
  const int* phase_patches;     // cluster q sweeps patch phase_patches[q]
  const int* slab;              // slab height (slow indices) per patch
  const int* pitch;             // shared-memory stride of a slow index per patch (>= its plane)
  const int* guard;             // zero floats before and after a CTA's extended slab, per patch
  const unsigned char* pool;    // item blocks, ordered by (phase, k, r, colour, item)
  // per region (direction, phase, k, r) = ((dir 2 + phase) K + k) csize + r, entries
  // [item_ptr[region], item_ptr[region + 1]), in sweep order:
  const int64_t* item_ptr;
  const int4* cmeta;            //   per item: rows, chunk, byte offset in the chunk, Rp | (last of its colour) << 30
  const int4* chunks;           //   per chunk (indexed like the items): pool offset (low, high word), bytes, -
  int max_items;                // most items of a region (shared-memory meta: 32 B each)
  int off_buf, off_mbar, off_meta;  // shared-memory layout (u slab at 0; 2 mbarriers; meta)
  const PatchMeta* patches;
  double* u;
  int* err;
};
// whether a cluster of csize CTAs of `threads` threads (tpr per row) with smem bytes fits the GPU (gs_staged.cu)
bool gs_staged_fits(int d, int p, int tpr, int csize, int smem, int threads);
cudaError_t launch_gs_staged(int d, int p, int nclusters, int smem, cudaStream_t st, const GsStagedArgs& a);
// xent: the nx entries of [e0, e0 + n) with couplings to the other parity
void launch_wait_expiry_probe(long long limit, cudaStream_t st, int* err, long long* elapsed_ns);
void launch_gs_fill_phase(int e0, int n, int nx, const int* xent, cudaStream_t st, const int64_t* f_off,
                          const int64_t* gs_pos, const int2* xrange, const int64_t* x_col, const double* x_val,
                          const double* f, const double* u, unsigned char* pool);

void launch_band(int d, int p, int mode, int ntiles, cudaStream_t st, const Tile* tiles, const PatchMeta* pm,
                 const double* band, int64_t nloc, const double* u, const double* f, double* out);
// out = f - A u with FP32 coefficients (band32: nb x nloc + 4 floats) and FP32 arithmetic
// g: threads per row group (1, 2, 4; other values: the built-in rule)
void launch_band_residual_f32(int d, int p, int ntiles, cudaStream_t st, const Tile* tiles, const PatchMeta* pm,
                              const float* band32, int64_t nloc, const double* u, const double* f, double* out,
                              int g = 0);
void launch_cross(int mode, int nx, cudaStream_t st, const int64_t* x_row, const int* x_ptr, const int64_t* x_col,
                  const double* x_val, const double* u, double* out);
void launch_shared(int nsh, cudaStream_t st, const int* sh_ptr, const int64_t* sh_pos, double* v, const double* f,
                   int mode);
// f32: FP32 arithmetic (inside the mixed-precision cycle), else FP64
void launch_restrict(int d, bool f32, int ntiles, cudaStream_t st, const Tile* tiles, const PatchMeta* pc,
                     const PatchMeta* pf, const XferMeta* xm, const int* ch_start, const double* ch_val, int cw,
                     const double* r, const double* w, const int* c_l2g, double* out);
void launch_prolong(int d, bool f32, int ntiles, cudaStream_t st, const Tile* tiles, const PatchMeta* pf,
                    const PatchMeta* pc, const XferMeta* xm, const int* par_start, const double* par_val, int pw,
                    const double* e, double* u);
// mode-wise 2D transfers: one CTA per block (patch, first row, end row) of output rows along xi_1,
// the intermediate of the xi_0 pass in smem bytes of shared memory (at most kXferSmemMax)
constexpr int kXferSmemMax = 96 * 1024;
cudaError_t prepare_transfers_mw2();
void launch_restrict_mw2(bool f32, int nblocks, int smem, cudaStream_t st, const int4* blocks, const PatchMeta* pc,
                         const PatchMeta* pf, const XferMeta* xm, const int* ch_start, const double* ch_val, int cw,
                         const double* r, const double* w, const int* c_l2g, double* out);
void launch_prolong_mw2(bool f32, int nblocks, int smem, cudaStream_t st, const int4* blocks, const PatchMeta* pf,
                        const PatchMeta* pc, const XferMeta* xm, const int* par_start, const double* par_val, int pw,
                        const double* e, double* u);
// arith 0: FP64 arithmetic (32 x 32 tiles), 1: FP32 arithmetic (64 x 64 tiles)
int gemm_tile(int arith);
// fused fast diagonalisation of small 2D patch interiors: one CTA per patch
constexpr int kFdSmallSmem = 200 * 1024;
// chunk buffers of the streamed Gauss-Seidel phase: two (one copy in flight
// while one is read) measured fastest; more buffers mean smaller chunks, and
// bulk copies of one SM complete one after another with a fixed cost each
constexpr int kGsRing = 2;
constexpr int kGsRingMax = 8;
// polls of a bounded mbarrier wait before it gives up: a failed poll suspends
// ~3.8 us on a GB300 (measured with the wait-expiry check), so ~1 s
constexpr long long kMbarPolls = 1ll << 18;
int fd_small_smem(int n0, int n1, bool f32);  // shared memory of one patch (must be <= kFdSmallSmem)
cudaError_t prepare_fd_small();
void launch_fd_small(int npatch, int smem, bool f32, cudaStream_t st, const FdSmall* patches, const double* r,
                     double* u, double tau);
// fused fast diagonalisation of 2D patch interiors on the FP32 path by one thread-block cluster per
// patch (fd_cluster.cu): cs CTAs per patch, each owning wm (>= ceil(n0 / cs), a multiple of 4)
// columns of the intermediates, ks groups of threads over the contraction index
struct FdClusterShape {
  int cs, wm, ks, threads, smem;
  int resident;  // clusters of this shape resident at once on the device
};
// the shape for interiors up to n0max x n1max (npatch clusters in a launch); false if none fits
bool fd_cluster_shape(int n0max, int n1max, int npatch, FdClusterShape* out);
cudaError_t launch_fd_cluster(int npatch, const FdClusterShape& s, cudaStream_t st, const FdSmall* patches,
                              const double* r, double* u, double tau);
cudaError_t prepare_gemm();  // shared-memory attributes of the SIMT GEMM (once per process)
// tA: element type of A in the step (0 double, 1 float); B is of the arithmetic type
void launch_gemm(int nitems, int arith, int tA, cudaStream_t st, const GemmTask* tasks, const GemmItem* items);
// tensor-core tiles (128 x 64, items built with these tile sizes): kind 0 TF32, 1 BF16
void launch_gemm_umma(int nitems, int kind, cudaStream_t st, const GemmTask* tasks, const GemmItem* items, int* err);
cudaError_t prepare_gemm_umma();
// TF32 on the tensor cores with FP32 operands (A, B of every task float): asynchronous element
// copies into the core-matrix layout, four slabs in flight
void launch_gemm_umma_tf32(int nitems, cudaStream_t st, const GemmTask* tasks, const GemmItem* items, int* err);
void launch_to_f32(int64_t n, cudaStream_t st, const double* x, float* y);
// interiors of the patches of r as compact FP32 row blocks (TF32 contractions with 16-byte copies)
void launch_gather_interior_f32(int npatch, int64_t total, cudaStream_t st, const int64_t* e_ptr,
                                const int64_t* ibase, const int* n0s, const int* N0s, const int64_t* d_off,
                                const int* d_ld, const double* r, float* dst);
// zpool: double, or float when zf32 (the interface pieces of the mixed-precision smoother)
void launch_piece(int nitems, int max_n, cudaStream_t st, const PieceItem* items, const PieceMeta* pieces,
                  const void* zpool, bool zf32, const int64_t* piece_pos, const double* r, double* u, double tau,
                  int mode);
cudaError_t prepare_piece_kernel(int max_n);
void launch_dot(int64_t n, cudaStream_t st, const double* a, const double* b, const double* w, double* partials,
                double* scal, unsigned int* counter, int slot, int op);
void launch_cg_xr(int64_t n, cudaStream_t st, double* x, double* r, const double* p, const double* q,
                  const double* w, double* partials, double* scal, unsigned int* counter);
void launch_cg_p(int64_t n, cudaStream_t st, double* p, const double* z, const double* scal);
// device-driven PCG loop: control kernels that set the conditions of the loop's graph nodes
// (handles are cudaGraphConditionalHandle values)
void launch_cg_ctl_a(cudaStream_t st, const double* scal, CgLoopState* state, double* hist,
                     unsigned long long hloop, unsigned long long hconf, unsigned long long hcont);
void launch_cg_ctl_c(cudaStream_t st, const double* scal, CgLoopState* state, double* hist,
                     unsigned long long hloop, unsigned long long hcont);
void launch_cg_ctl_0(cudaStream_t st, double* scal, CgLoopState* state, double* hist, unsigned long long hzero,
                     unsigned long long hgo, unsigned long long hloop);
// tolerance and iteration limit of the next device-driven solve (nf > 0: also ||f||), state reset
void launch_cg_loop_init(cudaStream_t st, double* scal, CgLoopState* state, double tol, double nf, int maxit);
void launch_scatter(int64_t nloc, cudaStream_t st, const int* l2g, const double* g, double* loc);
void launch_gather(int ndof, cudaStream_t st, const int64_t* owner, const double* loc, double* g);
void launch_axpby(int64_t n, cudaStream_t st, double a, const double* x, double b, double* y);
int red_blocks();
// kernels enqueued by this host thread so far
long long launch_counter();
void count_launch();  // for launchers outside kernels.cu
// fused 2D fast diagonalisation on the tensor cores (fd_fused.cu): two launches (pass 0, pass 1)
// of one CTA per FdFusedTask; interiors up to fd_fused_max_rows() rows (n1)
int fd_fused_smem(int mt);  // dynamic shared memory of tasks with mt 128-row tiles
int fd_fused_max_rows();
cudaError_t prepare_fd_fused();
void launch_fd_fused(int ntasks, int smem, cudaStream_t st, const FdFusedTask* tasks, double tau, int* err);

}  // namespace dev
}  // namespace mgiga
