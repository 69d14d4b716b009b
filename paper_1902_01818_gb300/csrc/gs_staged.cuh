// a4 on the mixed path: the patch-parallel multicolour Gauss-Seidel phase (Sec. 4, Algorithm 2), one
// thread-block cluster per patch, the CTA's rows of each colour staged through shared memory by bulk
// asynchronous copies.  The kernel template; gs_staged_2d.cu and gs_staged_3d.cu instantiate it per
// degree and threads per row (two translation units, compiled side by side).
#pragma once

#include <cstdint>

#include <cooperative_groups.h>

#include "device.cuh"
#include "kernels.h"
#include "ptx.cuh"

namespace mgiga {
namespace dev {

// ---------------------------------------------------------------------------
// Base colours of one patch parity, mixed path (FP32 arithmetic).  The patch
// is split along its slowest direction into the slabs of the CTAs of one
// cluster; a CTA keeps u of its slab plus P slow indices on each side (the
// halo, refreshed by its neighbours through distributed shared memory) in
// shared memory, with zero rows beyond the patch and zero guards at both
// ends, so that every band neighbour of a row is a plain shared-memory read
// (off-patch columns have zero coefficients).  For every colour the CTA's
// rows come as one or more contiguous blocks ("items") -- FP32 coefficients
// [line][row][o_0], the packed slab position, f minus the couplings to the other
// parity (written by gs_fill_phase before the launch) and the inverse
// diagonal; consecutive items are fetched together as one bulk asynchronous
// copy ("chunk"), two chunk buffers in flight, mbarrier completion.  Colours are separated by the
// CTA barrier; where the residue of the slow index changes from one colour to the next, by the
// hardware cluster barrier, which publishes the halo stores (no row of a run of colours with one
// slow residue reads a halo value that a neighbour updates during the run).
// Every wait on an mbarrier is bounded: on expiry the CTA records the error,
// stops computing and keeps taking part in the barriers.
// ---------------------------------------------------------------------------
template <int D, int P, int TPR>
__global__ void __launch_bounds__(1024, 1) gs_patch_staged(GsStagedArgs a) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int W = 2 * P + 1;
  constexpr int NOB = D == 2 ? W : W * W;
  constexpr int NB = NOB * W;
  cg::cluster_group cluster = cg::this_cluster();
  const int cs = a.csize;
  const int q = blockIdx.x / cs;
  const int r = (int)cluster.block_rank();
  const int k = a.phase_patches[q];
  const int S = a.slab[k];
  const int pitch = a.pitch[k];  // shared-memory stride of one slow index (>= plane)
  const int G = a.guard[k];      // zero floats before and after the extended slab
  const PatchMeta pm = a.patches[k];
  const int N0 = pm.N[0];
  const int plane = D == 2 ? N0 : N0 * pm.N[1];
  const int nslow = D == 2 ? pm.N[1] : pm.N[2];
  const int s_lo = r * S, s_hi = min(nslow, (r + 1) * S);
  const int ext_len = 2 * G + (S + 2 * P) * pitch;  // slow indices s_lo - P .. s_lo + S + P - 1
  const int H = (P + S - 1) / S;  // CTAs on each side whose halo may hold my indices
  float* us = reinterpret_cast<float*>(smem);
  unsigned char* const buf0 = smem + a.off_buf;
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smem + a.off_mbar);
  int4* cm = reinterpret_cast<int4*>(smem + a.off_meta);  // per item: rows, chunk, offset in chunk, Rp | end flags
  int4* ch = cm + a.max_items;                             // per chunk: byte offset (lo, hi), bytes, -
  const int tid = threadIdx.x;
  const int nthr = blockDim.x;
  const int dir = a.forward ? 0 : 1;
  const int ph = a.c_begin / a.base;
  const int64_t reg = (((int64_t)dir * 2 + ph) * a.K + k) * cs + r;
  const int64_t ibase = a.item_ptr[reg];
  const int nc = (int)(a.item_ptr[reg + 1] - ibase);  // items (sub-blocks of colours) in sweep order
  for (int i = tid; i < nc; i += nthr) {
    cm[i] = a.cmeta[ibase + i];
    ch[i] = a.chunks[ibase + i];
  }
  const int nbuf = a.nbuf;  // ring of chunk buffers: chunk j in buffer j % nbuf
  if (tid == 0) {
    for (int b = 0; b < nbuf; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[b])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int nchunk = nc > 0 ? cm[nc - 1].y + 1 : 0;
  int issued = 0;  // thread 0: chunks 0 .. issued - 1 have been requested
  auto copy = [&](int j) {  // thread 0: chunk j into its buffer
    const int b = j % nbuf;
    const unsigned bar = smem_u32(&mbar[b]);
    const int4 c = ch[j];
    const int64_t off = (int64_t)(unsigned)c.x | ((int64_t)c.y << 32);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(c.z) : "memory");
    if (c.z > 0)
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_u32(buf0 + (size_t)b * a.cap)),
          "l"(a.pool + off), "r"(c.z), "r"(bar)
          : "memory");
    issued = j + 1;
  };
  if (tid == 0)
    for (int j = 0; j < min(nbuf, nchunk); ++j) copy(j);
  // u of the extended slab (zero outside the patch and in the guards), four independent loads per thread
  {
    const double* ug = a.u + pm.off;
    const int body = (S + 2 * P) * pitch;
    for (int i0 = tid; i0 < ext_len; i0 += 4 * nthr) {
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int i = i0 + j * nthr;
        v[j] = 0.0f;
        const int t = i - G;
        if (i < ext_len && t >= 0 && t < body) {
          const int row = t / pitch, col = t - row * pitch;
          const int s = s_lo - P + row;
          if (s >= 0 && s < nslow && col < plane) v[j] = (float)__ldcg(ug + (int64_t)s * plane + col);
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (i0 + j * nthr < ext_len) us[i0 + j * nthr] = v[j];
    }
  }
  // one CTA per patch: the CTA barrier orders everything; else the cluster
  // barrier (release/acquire) also publishes the halo stores, and here keeps
  // neighbours from refreshing a halo before it is loaded
  auto sync_all = [&]() {
    if (cs == 1) __syncthreads();
    else cluster.sync();
  };
  sync_all();
  // TPR: threads per row (power of two, 4..32), a compile-time constant so that the row's line loop
  // and its shuffle tree unroll
  const int lane = tid & 31;
  const int sub = lane & (TPR - 1);
  const int warp = tid >> 5;
  const int rows_per_warp = 32 / TPR;
  const int rows_per_cta = nthr / TPR;
  bool ok = true;
  bool synced = true;  // no item has been read since the last barrier
  int cur = -1;
  int failed_at = -1;  // the chunk whose wait expired
  for (int ci = 0; ci < nc; ++ci) {
    // rows, chunk, offset in chunk, Rp | (last item of its colour) << 30 | (last of its slow-residue run) << 29
    const int4 m = cm[ci];
    const int b = m.y % nbuf;
    if (m.y != cur) {  // first item of chunk m.y
      // chunk m.y + nbuf - 1 goes into the buffer of chunk m.y - 1: every thread must be done
      // with it (a colour split across two chunks has no barrier between its items)
      if (!synced) __syncthreads();
      cur = m.y;
      const unsigned parity = (unsigned)((m.y / nbuf) & 1);
      if (ok && !mbar_wait(smem_u32(&mbar[b]), parity)) {
        ok = false;
        failed_at = m.y;
        atomicExch(a.err, 2);
      }
      if (tid == 0 && ok && nbuf >= 2 && m.y >= 1 && m.y + nbuf - 1 < nchunk) copy(m.y + nbuf - 1);
    }
    const int R = m.x, Rp = m.w & ((1 << 29) - 1);
    const float* coef = reinterpret_cast<const float*>(buf0 + (size_t)b * a.cap + m.z);
    const int* lidx = reinterpret_cast<const int*>(coef + NB * Rp);
    const float* fv = reinterpret_cast<const float*>(lidx + Rp);
    const float* dinv = fv + Rp;
    if (ok) {
      for (int base = warp * rows_per_warp; base < R; base += rows_per_cta) {
        const int row = base + lane / TPR;
        const bool active = row < R;
        float acc = 0.0f, acc1 = 0.0f;  // two chains of dependent FMAs
        int own = 0, srow = 0, rest = 0;
        if (active) {
          const unsigned li = (unsigned)lidx[row];  // (slow index - s_lo) << 20 | index within the plane
          srow = (int)(li >> 20);
          rest = (int)(li & 0xFFFFFu);
          own = G + (srow + P) * pitch + rest;
#pragma unroll(D == 2 ? 16 : 4)
          for (int ob = sub; ob < NOB; ob += TPR) {
            const int o1 = ob % W, o2 = ob / W;
            const float* ur = us + own + (D == 2 ? (o1 - P) * pitch : (o2 - P) * pitch + (o1 - P) * N0) - P;
            const float* cr = coef + (ob * Rp + row) * W;  // the row's line, 2P + 1 contiguous floats
#pragma unroll
            for (int o0 = 0; o0 < W; ++o0) {
              if (o0 & 1) acc1 = fmaf(cr[o0], ur[o0], acc1);
              else acc = fmaf(cr[o0], ur[o0], acc);
            }
          }
        }
        acc += acc1;
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (active && sub == 0) {
          const float v = us[own] + (fv[row] - acc) * dinv[row];
          us[own] = v;
          // refresh the copies of this value in the neighbours' halos
          if (H == 1) {  // slabs at least P thick: only the first / last P slow indices are halo rows
            if (srow < P && r > 0) cluster.map_shared_rank(us, r - 1)[G + (srow + S + P) * pitch + rest] = v;
            if (srow >= S - P && r + 1 < cs) cluster.map_shared_rank(us, r + 1)[G + (srow - S + P) * pitch + rest] = v;
          } else {
            const int s = s_lo + srow;
            for (int rr = max(0, r - H); rr <= min(cs - 1, r + H); ++rr) {
              const int lo2 = rr * S - P;
              if (rr == r || s < lo2 || s >= lo2 + S + 2 * P) continue;
              float* rem = cluster.map_shared_rank(us, rr);
              rem[G + (s - lo2) * pitch + rest] = v;
            }
          }
        }
      }
    }
    // rows of one colour never couple: a barrier after its last item only; the
    // halos change only between runs of colours with one residue of the slow index
    if (m.w & (1 << 29)) sync_all();
    else if (m.w & (1 << 30)) __syncthreads();
    synced = (m.w & (1 << 30)) != 0;
  }
  // after an expired wait: let the copies still in flight land (bounded) before the CTA exits
  if (!ok && tid == 0)
    for (int j = failed_at; j < issued; ++j) mbar_wait(smem_u32(&mbar[j % nbuf]), (unsigned)((j / nbuf) & 1));
  // the slab back to global memory
  double* ug = a.u + pm.off;
  const int n_own = (s_hi - s_lo) * plane;
  for (int i = tid; i < n_own; i += nthr) {
    const int row = i / plane, col = i - row * plane;
    ug[(int64_t)(s_lo + row) * plane + col] = (double)us[G + (row + P) * pitch + col];
  }
}


// the kernel of (D, p, tpr), or nullptr
template <int D>
void* gs_staged_ptr_dim(int p, int tpr) {
#define MG_TPR(PP)                                              \
  case PP:                                                      \
    return tpr == 4 ? (void*)gs_patch_staged<D, PP, 4>          \
         : tpr == 8 ? (void*)gs_patch_staged<D, PP, 8>          \
         : tpr == 16 ? (void*)gs_patch_staged<D, PP, 16>        \
         : tpr == 32 ? (void*)gs_patch_staged<D, PP, 32> : nullptr;
  switch (p) {
    MG_TPR(1) MG_TPR(2) MG_TPR(3) MG_TPR(4) MG_TPR(5) MG_TPR(6) MG_TPR(7) MG_TPR(8)
    default: return nullptr;
  }
#undef MG_TPR
}
void* gs_staged_ptr_2d(int p, int tpr);  // gs_staged_2d.cu
void* gs_staged_ptr_3d(int p, int tpr);  // gs_staged_3d.cu

}  // namespace dev
}  // namespace mgiga
