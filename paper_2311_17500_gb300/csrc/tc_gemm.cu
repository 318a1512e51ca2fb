// Fast-diagonalization transforms on the 5th-generation tensor cores
// (tcgen05, TF32 inputs, FP32 accumulation in tensor memory).
//
// One transform contracts the contiguous axis b of a tensor [T][a][b] with an
// n_j x n_b matrix M and writes the result rotated, [T][j][a]:
//     out[(t n_j + j) A + a] = sum_k X[(t A + a) n_b + k] M[j][k],
// with the innermost part of a optionally padded in the output (row stride
// A_in_stride) so that the next transform can read it with TMA.  Seen as a
// GEMM, the rows (t, a) of X are K-major and so are the rows j of M.
// Rotating the output makes the next axis contiguous; after d transforms the
// original axis order is restored (Eq. factorized: U_s = U_d x ... x U_1
// applied axis by axis).
//
// Two kernels:
//  * tc_xform_tma (used whenever M fits in shared memory): warp-specialized.
//    Warp 0 loads M once and then streams 128-row x 32-column chunks of X
//    with TMA (cp.async.bulk.tensor, 128-byte swizzle) into an S-stage ring;
//    warp 1 issues tcgen05.mma (M = 128, N = round_up(n_j, 16), K = 8 per
//    instruction) into one of two TMEM accumulators and commits to mbarriers;
//    warps 4..7 read the accumulator (tcgen05.ld.32x32b) and store the rows
//    while the next tile is multiplied into the other accumulator.
//  * tc_xform_staged (fallback for larger M): all threads stage K-chunks of X
//    and M in the canonical no-swizzle layout, one thread issues the MMAs.
// Every mbarrier wait is bounded: a wait that gives up sets the error flag,
// the role stops, the CTA frees its tensor memory and returns.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <cstdint>
#include <cstring>
#include <vector>
#include <cuda.h>
#include <cudaTypedefs.h>
#include "st_internal.h"
#include "dev_sync.cuh"
#include "pdl.cuh"

namespace {

constexpr int kTcKC = 32;          // K columns per chunk (128 bytes of TF32 = one swizzle row)
constexpr int kTcRows = 128;       // MMA M (rows of X per tile)
constexpr long long kWaitLimit = 1ll << 22;


// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension
// byte offset (K direction, no-swizzle K-major only), stride-dimension byte
// offset (8-row groups), descriptor version 1, layout (0: no swizzle,
// 2: 128-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)(layout & 7u) << 61;
  return d;
}

// Instruction descriptor for kind::tf32: D = F32, A = B = TF32, both K-major,
// N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}


__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

// 16 consecutive TMEM columns of this thread's lane; the values are valid
// only after tmem_ld_wait().
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t *v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  tmem_ld16_nowait(taddr, v);
  tmem_ld_wait();
}

struct XformArgs {
  float *out;
  const float *X;
  const float *Mp;
  long long R;           // rows of X (t, a)
  long long in_stride;   // row stride of X (elements)
  int nb, nj, Npad, Kpad;
  long long Aa, A_inner, A_in_stride;   // a = a_outer * A_inner + a_inner; output row stride of a_inner
  int ncols_tmem;
  int *err;
};

// stores one accumulator row (16 columns starting at c0) of output row `row`
__device__ __forceinline__ void store_row16(const XformArgs &x, long long row, int c0, const uint32_t (&v)[16]) {
  if (row >= x.R) return;
  long long t = row / x.Aa, a = row - t * x.Aa;
  long long ao = a / x.A_inner, ai = a - ao * x.A_inner;
  long long A_outer = x.Aa / x.A_inner;
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    int j = c0 + u;
    if (j < x.nj) x.out[((t * x.nj + j) * A_outer + ao) * x.A_in_stride + ai] = __uint_as_float(v[u]);
  }
}

// ---------------------------------------------------------------- TMA kernel
template <int S>
__global__ void __launch_bounds__(256) tc_xform_tma_kernel(const __grid_constant__ CUtensorMap tmX,
                                                           const __grid_constant__ CUtensorMap tmB, XformArgs x) {
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte aligned region for the 128-byte swizzle pattern
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int nchunks = x.Kpad / kTcKC;
  const uint32_t bbytes_chunk = (uint32_t)x.Npad * 128u;       // one 32-column chunk of M
  const uint32_t sB = base;                                     // nchunks x Npad rows x 128 B
  const uint32_t sX = base + (uint32_t)nchunks * bbytes_chunk;  // S x 128 rows x 128 B
  __shared__ __align__(8) uint64_t full[S], empty[S], tdone[2], afree[2], bfull;
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  pdl_trigger();
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(x.ncols_tmem)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    fail = 0;
    for (int i = 0; i < S; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[i])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[i])) : "memory");
    }
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tdone[i])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&afree[i])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bfull)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const long long ntiles = (x.R + kTcRows - 1) / kTcRows;
  const long long my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const long long njobs = my_tiles * nchunks;
  const int acc_cols = x.ncols_tmem / 2;

  if (warp == 0 && lane == 0) {
    // ---- producer: M once, then the X chunks of every (tile, chunk) job
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bfull)),
                 "r"(bbytes_chunk * (uint32_t)nchunks)
                 : "memory");
    for (int c = 0; c < nchunks; ++c)
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
              "r"(sB + (uint32_t)c * bbytes_chunk),
          "l"((uint64_t)&tmB), "r"(c * kTcKC), "r"(0), "r"(smem_u32(&bfull))
          : "memory");
    pdl_wait();   // X is written by the previous kernel (M above is constant)
    for (long long q = 0; q < njobs; ++q) {
      const int st = (int)(q % S);
      const long long u = q / S;
      if (u >= 1 && !mbar_wait(smem_u32(&empty[st]), (uint32_t)((u - 1) & 1), kWaitLimit)) {
        fail = 1;
        break;
      }
      if (*(volatile int *)&fail) break;
      const long long tile = blockIdx.x + (q / nchunks) * gridDim.x;
      const int kc = (int)(q % nchunks) * kTcKC;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&full[st])),
                   "r"(kTcRows * 128)
                   : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
              "r"(sX + (uint32_t)st * (kTcRows * 128)),
          "l"((uint64_t)&tmX), "r"(kc), "r"((int)(tile * kTcRows)), "r"(smem_u32(&full[st]))
          : "memory");
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    const uint32_t idesc = tf32_idesc(kTcRows, x.Npad);
    bool ok = mbar_wait(smem_u32(&bfull), 0, kWaitLimit);
    if (!ok) fail = 1;
    for (long long q = 0; ok && q < njobs; ++q) {
      const int st = (int)(q % S);
      const long long u = q / S;
      const int chunk = (int)(q % nchunks);
      const long long i = q / nchunks;
      const int acc = (int)(i & 1);
      if (chunk == 0 && i >= 2 && !mbar_wait(smem_u32(&afree[acc]), (uint32_t)(((i >> 1) - 1) & 1), kWaitLimit)) {
        fail = 1;
        break;
      }
      if (!mbar_wait(smem_u32(&full[st]), (uint32_t)(u & 1), kWaitLimit)) {
        fail = 1;
        break;
      }
      if (*(volatile int *)&fail) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t xs = sX + (uint32_t)st * (kTcRows * 128);
      const uint32_t bs = sB + (uint32_t)chunk * bbytes_chunk;
#pragma unroll
      for (int s = 0; s < kTcKC / 8; ++s) {
        uint64_t ad = smem_desc(xs + 32 * s, 16, 1024, 2);
        uint64_t bd = smem_desc(bs + 32 * s, 16, 1024, 2);
        mma_tf32(tmem + (uint32_t)(acc * acc_cols), ad, bd, idesc, (chunk > 0 || s > 0) ? 1u : 0u);
      }
      mma_commit(smem_u32(&empty[st]));
      if (chunk == nchunks - 1) mma_commit(smem_u32(&tdone[acc]));
    }
  } else if (warp >= 4) {
    // ---- epilogue: warp w reads TMEM lanes 32 (w - 4) .. +31
    pdl_wait();   // the output may still be read by the previous kernel
    const int lw = warp - 4;
    for (long long i = 0; i < my_tiles; ++i) {
      const int acc = (int)(i & 1);
      if (!mbar_wait(smem_u32(&tdone[acc]), (uint32_t)((i >> 1) & 1), kWaitLimit)) {
        fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const long long tile = blockIdx.x + i * gridDim.x;
      const long long row = tile * kTcRows + lw * 32 + lane;
      // output address of this row's j = 0 and the stride between j (once per tile)
      const bool valid = row < x.R;
      float *obase = x.out;
      long long jstride = 0;
      if (valid) {
        const long long t = row / x.Aa, a = row - t * x.Aa;
        const long long ao = a / x.A_inner, ai = a - ao * x.A_inner;
        const long long A_outer = x.Aa / x.A_inner;
        jstride = A_outer * x.A_in_stride;
        obase = x.out + (t * x.nj * A_outer + ao) * x.A_in_stride + ai;
      }
      const uint32_t tl = tmem + ((uint32_t)(lw * 32) << 16) + (uint32_t)(acc * acc_cols);
      int c0 = 0;
      for (; c0 + 32 <= x.Npad; c0 += 32) {
        uint32_t v[32];
        tmem_ld16_nowait(tl + (uint32_t)c0, v);
        tmem_ld16_nowait(tl + (uint32_t)(c0 + 16), v + 16);
        tmem_ld_wait();
        if (valid) {
#pragma unroll
          for (int u = 0; u < 32; ++u)
            if (c0 + u < x.nj) obase[(long long)(c0 + u) * jstride] = __uint_as_float(v[u]);
        }
      }
      if (c0 < x.Npad) {
        uint32_t v[16];
        tmem_ld16(tl + (uint32_t)c0, v);
        if (valid) {
#pragma unroll
          for (int u = 0; u < 16; ++u)
            if (c0 + u < x.nj) obase[(long long)(c0 + u) * jstride] = __uint_as_float(v[u]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&afree[acc])) : "memory");
    }
  }
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(x.ncols_tmem) : "memory");
  }
  if (threadIdx.x == 0 && fail) atomicExch(x.err, 1);
}

// ---------------------------------------------------------------- staged kernel
// Stage a rows x KC chunk (columns kc .. kc+KC of a row-major source with row
// stride ld and valid extents nrows x ncols) into the canonical no-swizzle
// layout: byte offset ((r/8) (KC/4) + k/4) 128 + (r%8) 16 + (k%4) 4.
__device__ __forceinline__ void stage_chunk(float *dst, const float *src, long long row0, long long nrows,
                                            long long ld, int kc, int ncols, int rows) {
  constexpr int KG = kTcKC / 4;
  for (int idx = threadIdx.x; idx < rows * kTcKC; idx += blockDim.x) {
    int w = idx & 31, blk = idx >> 5;
    int rg = blk / KG, kg = blk - rg * KG;
    int r = rg * 8 + (w >> 2), k = kg * 4 + (w & 3);
    long long row = row0 + r;
    int kk = kc + k;
    dst[idx] = (row < nrows && kk < ncols) ? src[row * ld + kk] : 0.0f;
  }
}

__global__ void __launch_bounds__(128) tc_xform_staged_kernel(XformArgs x) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float *sX = reinterpret_cast<float *>(smem_raw);            // 128 x KC
  float *sB = sX + kTcRows * kTcKC;                            // Npad x KC
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(x.ncols_tmem)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t mb = smem_u32(&mbar);
  const uint32_t idesc = tf32_idesc(kTcRows, x.Npad);
  const uint32_t sbo = (kTcKC / 4) * 128;
  uint32_t phase = 0;
  const long long ntiles = (x.R + kTcRows - 1) / kTcRows;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long row0 = tile * kTcRows;
    for (int kc = 0; kc < x.Kpad; kc += kTcKC) {
      stage_chunk(sX, x.X, row0, x.R, x.in_stride, kc, x.nb, kTcRows);
      stage_chunk(sB, x.Mp, 0, x.Npad, x.Kpad, kc, x.Kpad, x.Npad);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int s = 0; s < kTcKC / 8; ++s) {
          uint64_t ad = smem_desc(smem_u32(sX) + 2 * s * 128, 128, sbo, 0);
          uint64_t bd = smem_desc(smem_u32(sB) + 2 * s * 128, 128, sbo, 0);
          mma_tf32(tmem, ad, bd, idesc, (kc > 0 || s > 0) ? 1u : 0u);
        }
        mma_commit(mb);
      }
      if (!mbar_wait(mb, phase, kWaitLimit)) fail = 1;
      phase ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      __syncthreads();
      if (fail) break;
    }
    if (fail) break;
    const long long row = row0 + warp * 32 + lane;
    for (int c0 = 0; c0 < x.Npad; c0 += 16) {
      uint32_t v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      store_row16(x, row, c0, v);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(x.ncols_tmem) : "memory");
  }
  if (threadIdx.x == 0 && fail) atomicExch(x.err, 1);
}

// The driver's tensor-map encoder, looked up once (thread-safe static
// initialization; null if the driver does not provide it).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
      cudaGetLastError();
      return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    }
    return (PFN_cuTensorMapEncodeTiled_v12000)p;
  }();
  return fn;
}

bool encode_2d(CUtensorMap *m, const float *ptr, long long inner, long long outer, long long stride_elems,
               int box_inner, int box_outer) {
  const PFN_cuTensorMapEncodeTiled_v12000 g_encode = tensor_map_encoder();
  if (!g_encode) return false;
  cuuint64_t gdim[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t gstride[1] = {(cuuint64_t)stride_elems * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)ptr, gdim, gstride, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int tc_ncols(int npad, int accs) {
  int c = 32;
  while (c < npad * accs) c <<= 1;
  return c;
}

}  // namespace

// One rotating transform on the tensor cores (see the file comment).
// X rows: R rows of nb values with stride in_stride; output rows of a_inner
// with stride A_in_stride.  Requires nj <= 256.
st_status launch_tc_xform(cudaStream_t s, float *out, const float *X, long long R, int nb, long long in_stride,
                          const float *Mpad, int nj, int Npad, int Kpad, long long Aa, long long A_inner,
                          long long A_in_stride, int *err) {
  if (Npad > 256 || Npad % 16 != 0 || Kpad % kTcKC != 0 || R <= 0) return ST_ERR_ARG;
  XformArgs x;
  x.out = out; x.X = X; x.Mp = Mpad; x.R = R; x.in_stride = in_stride;
  x.nb = nb; x.nj = nj; x.Npad = Npad; x.Kpad = Kpad;
  x.Aa = Aa; x.A_inner = A_inner; x.A_in_stride = A_in_stride; x.err = err;
  const long long ntiles = (R + kTcRows - 1) / kTcRows;
  constexpr int S = 4;
  size_t need_tma = (size_t)Npad * Kpad * 4 + (size_t)S * kTcRows * 128 + 1024;
  bool aligned = ((uintptr_t)X % 16 == 0) && (in_stride % 4 == 0) && ((uintptr_t)Mpad % 16 == 0);
  CUtensorMap tmX, tmB;
  if (need_tma <= 200 * 1024 && aligned && encode_2d(&tmX, X, nb, R, in_stride, kTcKC, kTcRows) &&
      encode_2d(&tmB, Mpad, Kpad, Npad, Kpad, kTcKC, Npad)) {
    static std::atomic<unsigned long long> attr{0};
    ST_CUDA(smem_optin(tc_xform_tma_kernel<S>, 210 * 1024, attr));
    x.ncols_tmem = tc_ncols(Npad, 2);
    int grid = (int)std::min<long long>(ntiles, 152);
    st_count_launch();
    ST_CUDA(pdl_launch(tc_xform_tma_kernel<S>, dim3(grid), dim3(256), need_tma, s, tmX, tmB, x));
    ST_CUDA(cudaGetLastError());
    return ST_OK;
  }
  x.ncols_tmem = tc_ncols(Npad, 1);
  size_t need = (size_t)(kTcRows + Npad) * kTcKC * sizeof(float);
  int max_ctas = 512 / x.ncols_tmem;
  size_t floor_bytes = (size_t)(227 * 1024) / (size_t)(max_ctas + 1) + 1024;
  size_t sh = std::max(need, floor_bytes);
  static std::atomic<unsigned long long> attr_set{0};
  ST_CUDA(smem_optin(tc_xform_staged_kernel, 200 * 1024, attr_set));
  int grid = (int)std::min<long long>(ntiles, 152LL * max_ctas);
  st_count_launch();
  tc_xform_staged_kernel<<<grid, 128, sh, s>>>(x);
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}

namespace {
std::atomic<int> g_tc_state{0};
double g_tc_err = 0.0;
std::mutex g_tc_mutex;   // one self-test at a time (handles may be set up from several threads)

// host-side deterministic fill (linear congruential, values in [-1, 1))
void fill(std::vector<float> &v, unsigned seed) {
  unsigned xs = seed;
  for (auto &e : v) {
    xs = xs * 1664525u + 1013904223u;
    e = (float)((xs >> 8) * (1.0 / 8388608.0) - 1.0);
  }
}
}  // namespace

// One-time check of the tensor-core transform against the CUDA-core transform
// on a ragged problem (rows not a multiple of the tile, n not a multiple of
// 16), with a padded input row stride and a padded output as in the
// preconditioner.
int tc_state(cudaStream_t s, double *err_out) {
  if (g_tc_state.load() != 0) {
    std::lock_guard<std::mutex> lk(g_tc_mutex);
    if (err_out) *err_out = g_tc_err;
    return g_tc_state.load();
  }
  std::lock_guard<std::mutex> lk(g_tc_mutex);
  if (g_tc_state.load() != 0) {   // another thread finished the test meanwhile
    if (err_out) *err_out = g_tc_err;
    return g_tc_state.load();
  }
  int dev = 0, major = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (major != 10) {
    g_tc_state = -1;
    return -1;
  }
  const int nb = 131, nj = 131, T = 27, ld = 132;
  const long long Aa = 37, R = T * Aa, Apad = 40;
  const int Npad = 144, Kpad = 160;
  std::vector<float> X((size_t)R * ld, 0.0f), Xc((size_t)R * nb), M((size_t)nj * nb), Mp((size_t)Npad * Kpad, 0.0f);
  fill(Xc, 12345u);
  fill(M, 777u);
  for (long long r = 0; r < R; ++r)
    for (int k = 0; k < nb; ++k) X[(size_t)r * ld + k] = Xc[(size_t)r * nb + k];
  for (int j = 0; j < nj; ++j)
    for (int k = 0; k < nb; ++k) Mp[(size_t)j * Kpad + k] = M[(size_t)j * nb + k];
  float *dX = nullptr, *dXc = nullptr, *dM = nullptr, *dMp = nullptr, *d1 = nullptr, *d2 = nullptr;
  int *derr = nullptr;
  size_t no = (size_t)T * nj * Aa, nop = (size_t)T * nj * Apad;
  bool ok = cudaMalloc(&dX, X.size() * 4) == cudaSuccess && cudaMalloc(&dXc, Xc.size() * 4) == cudaSuccess &&
            cudaMalloc(&dM, M.size() * 4) == cudaSuccess && cudaMalloc(&dMp, Mp.size() * 4) == cudaSuccess &&
            cudaMalloc(&d1, nop * 4) == cudaSuccess && cudaMalloc(&d2, no * 4) == cudaSuccess &&
            cudaMalloc(&derr, 4) == cudaSuccess;
  double err = 1.0;
  if (ok) {
    cudaMemcpy(dX, X.data(), X.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(dXc, Xc.data(), Xc.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(dM, M.data(), M.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(dMp, Mp.data(), Mp.size() * 4, cudaMemcpyHostToDevice);
    cudaMemset(derr, 0, 4);
    cudaMemset(d1, 0, nop * 4);
    launch_rot_gemm<float>(s, d2, dXc, dM, nb, nj, Aa, T);
    st_status st = launch_tc_xform(s, d1, dX, R, nb, ld, dMp, nj, Npad, Kpad, Aa, Aa, Apad, derr);
    int herr = 1;
    if (st == ST_OK && cudaStreamSynchronize(s) == cudaSuccess) {
      cudaMemcpy(&herr, derr, 4, cudaMemcpyDeviceToHost);
      std::vector<float> o1(nop), o2(no);
      cudaMemcpy(o1.data(), d1, nop * 4, cudaMemcpyDeviceToHost);
      cudaMemcpy(o2.data(), d2, no * 4, cudaMemcpyDeviceToHost);
      double mx = 0.0, md = 0.0;
      for (long long t = 0; t < T; ++t)
        for (int j = 0; j < nj; ++j)
          for (long long a = 0; a < Aa; ++a) {
            double ref = o2[((size_t)t * nj + j) * Aa + a];
            double got = o1[((size_t)t * nj + j) * Apad + a];
            mx = std::max(mx, std::fabs(ref));
            double dd = std::fabs(got - ref);
            md = (dd == dd) ? std::max(md, dd) : 1e30;
          }
      err = mx > 0 ? md / mx : 1.0;
      if (herr) err = 1.0;
    }
    cudaGetLastError();
  }
  cudaFree(dX); cudaFree(dXc); cudaFree(dM); cudaFree(dMp); cudaFree(d1); cudaFree(d2); cudaFree(derr);
  g_tc_err = err;
  const int state = (ok && err < 5e-3) ? 1 : -1;
  g_tc_state = state;
  if (err_out) *err_out = err;
  return state;
}
