// a2 on the tensor cores for 2D patch interiors (Sec. 5, Eq. Ldef): the four
// contractions of the fast diagonalisation
//     X = (U_1^T R U_0) / (sigma + lambda_1 + lambda_0),   u += tau U_1 X U_0^T
// as two launches, each CTA chaining two contractions: it computes the
// n1 x 32 column block T = Rin Rt[:, cb] (all rows, on the tensor cores, the
// accumulator in tensor memory), moves T into shared memory as the operand of
// the second product and computes the 128 x 32 output tile L[rb, :] T with the
// epilogue of its pass (FdFusedTask).  The first product is recomputed by each
// of the ceil(n1 / 128) row tiles of a column block; in exchange the
// intermediate never leaves the SM and two launches replace four.
//
// Staging: 16-byte asynchronous copies into the K-major, non-swizzled
// core-matrix layout (8 rows x 16 bytes per core matrix), slabs of 16 FP32
// along K, three slabs in flight; one thread issues tcgen05.mma (kind::tf32,
// M = 128, N = 32, K = 8) and commits to the slab's mbarrier, which tells when
// the slab's buffer may be refilled.  Every mbarrier wait is bounded: on
// expiry the CTA records MGIGA_ETIMEOUT's flag, stops issuing MMAs, waits once
// more (bounded) for those in flight and frees its tensor memory.
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"
#include "ptx.cuh"

namespace mgiga {
namespace dev {

constexpr int FF_N = 32;                      // output columns per CTA: N of both products
constexpr int FF_KS = 16;                     // K elements per staged slab (64 bytes of a row)
constexpr int FF_ST = 3;                      // slabs in flight
constexpr int FF_LBO = 160;                   // core matrices along K 160 B apart: the eight 16-byte
                                              // copies of two rows land in distinct bank groups
constexpr int FF_SBO = (FF_KS / 4) * FF_LBO;  // 8-row groups 640 B apart
constexpr int FF_TLBO = 144;                  // T: core matrices along K 144 B apart (a warp's scalar
                                              // stores of 32 consecutive K hit 32 banks)
constexpr int FF_MT_MAX = 4;                  // 128-row tiles of the first product: n1 <= 512

__host__ __device__ constexpr int ff_sbo_t(int mt) { return (mt * 128 / 4) * FF_TLBO; }

int fd_fused_smem(int mt) {
  const int phase1 = FF_ST * (mt * 16 * FF_SBO + (FF_N / 8) * FF_SBO);
  const int phase2 = (FF_N / 8) * ff_sbo_t(mt) + FF_ST * 16 * FF_SBO;
  return phase1 > phase2 ? phase1 : phase2;
}

int fd_fused_max_rows() { return FF_MT_MAX * 128; }

__device__ __forceinline__ uint64_t ff_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);       // start address
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;   // leading byte offset: next core matrix along K
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;   // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                        // descriptor version (tcgen05); no swizzle
  return d;
}

// D = F32, A = B = TF32, both K-major; N >> 3 at bit 17, M >> 4 at bit 24
constexpr unsigned kFfIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(FF_N >> 3) << 17) |
                              ((unsigned)(128 >> 4) << 24);

// rows [row0, row0 + nrows) x K [k0, k0 + 16) of a row-major FP32 matrix into one slab; rows at or
// beyond rvalid and K at or beyond kvalid read as zero (16-byte chunks: the pitch pads K to 4)
__device__ __forceinline__ void ff_stage(unsigned char* dst, const float* src, int64_t ld, int row0, int nrows,
                                         int rvalid, int k0, int kvalid) {
  for (int e = threadIdx.x; e < nrows * 4; e += blockDim.x) {
    const int r = e >> 2, q = e & 3;
    const int row = row0 + r, k = k0 + 4 * q;
    const bool ok = row < rvalid && k < kvalid;
    const float* s = ok ? src + (int64_t)row * ld + k : src;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                     smem_u32(dst + (r >> 3) * FF_SBO + q * FF_LBO + (r & 7) * 16)),
                 "l"(s), "r"(ok ? 16 : 0)
                 : "memory");
  }
}

__device__ __forceinline__ void ff_mma(unsigned tmem_d, uint64_t ad, uint64_t bd, unsigned acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(kFfIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void ff_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void ff_ld16(unsigned taddr, float* v) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// One pipelined product over K = nk elements: for every slab the caller's `stage(slab, buffer)`
// enqueues the copies, `issue(slab, buffer)` (thread 0) the MMAs; bars[b] tracks buffer b.
// Returns false when a bounded wait expired (no further MMAs are issued then).
template <class Stage, class Issue>
__device__ __forceinline__ bool ff_pipeline(int nk, unsigned long long* bars, bool ok, int* err, Stage stage,
                                            Issue issue) {
  const int nst = (nk + FF_KS - 1) / FF_KS;
  for (int s = 0; s < FF_ST - 1; ++s) {
    if (s < nst) stage(s, s);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  for (int s = 0; s < nst; ++s) {
    const int b = s % FF_ST;
    asm volatile("cp.async.wait_group %0;" ::"n"(FF_ST - 2) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // copies -> tensor-core operand reads
    __syncthreads();
    if (threadIdx.x == 0 && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      issue(s, b);
      ff_commit(&bars[b]);
    }
    const int nxt = s + FF_ST - 1;
    if (nxt < nst) {
      if (s >= 1) {  // the buffer of slab s - 1 is refilled once its MMAs are done
        const int t = s - 1;
        if (ok && !mbar_wait(smem_u32(&bars[t % FF_ST]), (unsigned)((t / FF_ST) & 1))) {
          ok = false;
          atomicExch(err, 3);
        }
      }
      stage(nxt, nxt % FF_ST);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  // commits not consumed in the loop, in order (slab t is use t / FF_ST of its buffer)
  for (int t = max(0, nst - FF_ST); t < nst; ++t) {
    if (!mbar_wait(smem_u32(&bars[t % FF_ST]), (unsigned)((t / FF_ST) & 1))) {
      if (ok) atomicExch(err, 3);
      ok = false;
      mbar_wait(smem_u32(&bars[t % FF_ST]), (unsigned)((t / FF_ST) & 1));  // once more, bounded
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return ok;
}

__global__ void __launch_bounds__(256) fd_fused_tf32(const FdFusedTask* __restrict__ tasks, float tau, int* err) {
  extern __shared__ __align__(1024) unsigned char fsm[];
  __shared__ __align__(8) unsigned long long bars[2 * FF_ST];
  __shared__ unsigned tmem_slot;
  const FdFusedTask t = tasks[blockIdx.x];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = t.mt;
  // tensor memory: mt accumulators of T (32 columns each), then the output tile
  const unsigned need = (unsigned)((mt + 1) * FF_N);
  unsigned ncol = 32;
  while (ncol < need) ncol <<= 1;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ncol)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int b = 0; b < 2 * FF_ST; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[b])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_slot;

  // ---- first product: T (mt 128 x 32) = Rin (n1 x n0) Rt[:, cb], K = n0
  const int a1 = mt * 16 * FF_SBO;        // one slab of Rin (mt 128 rows)
  const int b1 = (FF_N / 8) * FF_SBO;     // one slab of Rt^T (32 rows)
  unsigned char* sA1 = fsm;
  unsigned char* sB1 = fsm + FF_ST * a1;
  const int n_lo = t.cb * FF_N;
  bool ok = ff_pipeline(
      t.n0, bars, true, err,
      [&](int s, int b) {
        ff_stage(sA1 + b * a1, t.rin, t.ldr, 0, mt * 128, t.n1, s * FF_KS, t.n0);
        ff_stage(sB1 + b * b1, t.bt, t.ldb, n_lo, FF_N, t.n0, s * FF_KS, t.n0);
      },
      [&](int s, int b) {
        const unsigned a0 = smem_u32(sA1 + b * a1), b0 = smem_u32(sB1 + b * b1);
#pragma unroll
        for (int j = 0; j < FF_KS / 8; ++j) {
          const uint64_t bd = ff_desc(b0 + 2 * FF_LBO * j, FF_LBO, FF_SBO);
          for (int i = 0; i < mt; ++i)
            ff_mma(tmem + (unsigned)(i * FF_N), ff_desc(a0 + i * 16 * FF_SBO + 2 * FF_LBO * j, FF_LBO, FF_SBO), bd,
                   (s > 0 || j > 0) ? 1u : 0u);
        }
      });

  // ---- T: tensor memory -> shared memory, as the K-major operand of the second product
  const int sbo_t = ff_sbo_t(mt);
  unsigned char* sT = fsm;                          // reuses the first product's buffers
  unsigned char* sA2 = fsm + (FF_N / 8) * sbo_t;    // slabs of L (128 rows)
  const int a2 = 16 * FF_SBO;
  ok = __syncthreads_and(ok);  // uniform from here: warp-collective loads and CTA barriers follow
  if (ok) {
    const int q = warp & 3, h = warp >> 2;  // TMEM lanes 32q.., columns 16h..
    for (int i = 0; i < mt; ++i) {
      float v[16];
      ff_ld16(tmem + ((unsigned)(q * 32) << 16) + (unsigned)(i * FF_N + h * 16), v);
      const int k = i * 128 + q * 32 + lane;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int n = h * 16 + c;
        *reinterpret_cast<float*>(sT + (n >> 3) * sbo_t + (k >> 2) * FF_TLBO + (n & 7) * 16 + (k & 3) * 4) = v[c];
      }
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic stores -> tensor-core reads
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // ---- second product: out (128 x 32) = L[rb rows, :] T, K = n1
  const unsigned tout = tmem + (unsigned)(mt * FF_N);
  const int m_lo = t.rb * 128;
  if (ok) ok = ff_pipeline(
      t.n1, bars + FF_ST, ok, err,
      [&](int s, int b) { ff_stage(sA2 + b * a2, t.lm, t.ldl, m_lo, 128, t.n1, s * FF_KS, t.n1); },
      [&](int s, int b) {
        const unsigned a0 = smem_u32(sA2 + b * a2), t0 = smem_u32(sT);
#pragma unroll
        for (int j = 0; j < FF_KS / 8; ++j)
          ff_mma(tout, ff_desc(a0 + 2 * FF_LBO * j, FF_LBO, FF_SBO),
                 ff_desc(t0 + (unsigned)((s * (FF_KS / 4) + 2 * j) * FF_TLBO), FF_TLBO, (unsigned)sbo_t),
                 (s > 0 || j > 0) ? 1u : 0u);
      });

  // ---- epilogue
  ok = __syncthreads_and(ok);
  if (ok) {
    const int q = warp & 3, h = warp >> 2;
    float v[16];
    ff_ld16(tout + ((unsigned)(q * 32) << 16) + (unsigned)(h * 16), v);
    const int m = m_lo + q * 32 + lane;
    const int nb = n_lo + h * 16;
    if (m < t.n1) {
      if (t.pass == 0) {
        float* x = t.xout + (int64_t)m * t.ldx;
        const float* dv = t.dinv + (int64_t)m * t.n0;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int n = nb + c;
          if (n < t.ldx) x[n] = n < t.n0 ? v[c] * dv[n] : 0.0f;
        }
      } else {
        double* u = t.u + t.ibase + (int64_t)m * t.N0;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int n = nb + c;
          if (n < t.n0) u[n] += (double)tau * (double)v[c];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncol) : "memory");
}

cudaError_t prepare_fd_fused() {
  return cudaFuncSetAttribute(fd_fused_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              fd_fused_smem(FF_MT_MAX));
}

void launch_fd_fused(int ntasks, int smem, cudaStream_t st, const FdFusedTask* tasks, double tau, int* err) {
  if (ntasks == 0) return;
  count_launch();
  fd_fused_tf32<<<ntasks, 256, smem, st>>>(tasks, (float)tau, err);
}

}  // namespace dev
}  // namespace mgiga
