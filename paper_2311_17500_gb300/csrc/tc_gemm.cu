// Fast-diagonalization transforms on the 5th-generation tensor cores
// (tcgen05, TF32 inputs, FP32 accumulation in tensor memory).
//
// One transform contracts the contiguous axis b of a tensor [T][a][b] with an
// n_j x n_b matrix M and writes the result rotated, [T][j][a]:
//     out[(t n_j + j) A + a] = sum_k X[(t A + a) n_b + k] M[j][k].
// Seen as a GEMM, the rows (t, a) of X are K-major (k contiguous), and so are
// the rows j of M, so both operands use the canonical K-major layout without
// swizzle: 8-row x 16-byte core matrices, LBO = 128 B between core matrices
// along K, SBO = (KC/4) * 128 B between 8-row groups.  Rotating the output
// makes the next axis contiguous; after d transforms the original axis order
// is restored (Eq. factorized: U_s = U_d x ... x U_1 is applied axis by axis).
//
// Each CTA (4 warps) owns a 128-row tile at a time: all threads stage K-chunks
// of the X tile and of M in shared memory, one thread issues tcgen05.mma with
// M = 128, N = round_up(n_j, 16), K = 8 per instruction into a TMEM
// accumulator and commits to an mbarrier; after the last chunk every warp
// reads its 32 TMEM lanes (tcgen05.ld.32x32b) and stores its rows.  Every
// mbarrier wait is bounded; a wait that gives up sets the error flag, the CTA
// stops taking tiles, frees its tensor memory and returns.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>
#include "st_internal.h"

namespace {

constexpr int kTcKC = 32;          // K columns staged per chunk (4 MMAs)
constexpr int kTcRows = 128;       // MMA M (rows of X per tile)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension
// byte offset (K direction for K-major), stride-dimension byte offset (8-row
// groups), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor for kind::tf32: D = F32, A = B = TF32, both K-major,
// N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t phase, long long limit) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Stage a rows x KC chunk (columns kc .. kc+KC of a row-major source with
// row stride ld and valid extents nrows x ncols) into the canonical layout:
// byte offset ((r/8) (KC/4) + k/4) 128 + (r%8) 16 + (k%4) 4.  Lanes of a warp
// write one contiguous 128-byte core matrix, so the stores are conflict-free.
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

__global__ void __launch_bounds__(128) tc_rot_gemm_kernel(float *__restrict__ out, const float *__restrict__ X,
                                                          const float *__restrict__ Mp, long long R, int nb, int nj,
                                                          int Npad, int Kpad, long long Aa, int ncols_tmem,
                                                          int *err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float *sX = reinterpret_cast<float *>(smem_raw);            // 128 x KC
  float *sB = sX + kTcRows * kTcKC;                            // Npad x KC
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ncols_tmem)
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
  const uint32_t idesc = tf32_idesc(kTcRows, Npad);
  const uint32_t sbo = (kTcKC / 4) * 128;
  uint32_t phase = 0;
  const long long ntiles = (R + kTcRows - 1) / kTcRows;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long row0 = tile * kTcRows;
    for (int kc = 0; kc < Kpad; kc += kTcKC) {
      stage_chunk(sX, X, row0, R, nb, kc, nb, kTcRows);
      stage_chunk(sB, Mp, 0, Npad, Kpad, kc, Kpad, Npad);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int s = 0; s < kTcKC / 8; ++s) {
          uint64_t ad = smem_desc(smem_u32(sX) + 2 * s * 128, 128, sbo);
          uint64_t bd = smem_desc(smem_u32(sB) + 2 * s * 128, 128, sbo);
          uint32_t acc = (kc > 0 || s > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\t"
              "setp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                     : "memory");
      }
      // the MMAs read sX / sB: wait for their completion before restaging
      if (!mbar_wait(mb, phase, 1ll << 22)) fail = 1;
      phase ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      __syncthreads();
      if (fail) break;
    }
    if (fail) break;
    // epilogue: TMEM lanes 32*warp .. +31 hold rows row0 + 32*warp + lane
    const long long row = row0 + warp * 32 + lane;
    long long t = 0, a = 0;
    if (row < R) {
      t = row / Aa;
      a = row - t * Aa;
    }
    for (int c0 = 0; c0 < Npad; c0 += 16) {
      uint32_t v[16];
      uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < R) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          int j = c0 + u;
          if (j < nj) out[(t * nj + j) * Aa + a] = __uint_as_float(v[u]);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols_tmem) : "memory");
  }
  if (threadIdx.x == 0 && fail) atomicExch(err, 1);
}

// Pipelined variant for transform matrices that fit in shared memory: the
// whole padded matrix M stays resident (canonical layout over all K), and the
// X chunks of 128 rows x KC stream through an S-stage ring filled with
// cp.async (zero-fill outside the tensor).  The sequence of (tile, chunk)
// jobs of a CTA is prefetched S-1 jobs ahead across tile boundaries, so the
// loads of the next tile overlap the MMAs and the epilogue of the current one.
// A stage is refilled only after the mbarrier of the MMAs that read it has
// completed; all waits are bounded.
template <int S>
__global__ void __launch_bounds__(256) tc_rot_gemm2_kernel(float *__restrict__ out, const float *__restrict__ X,
                                                           const float *__restrict__ Mp, long long R, int nb,
                                                           int nj, int Npad, int Kpad, long long Aa, int ncols_tmem,
                                                           int *err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float *sB = reinterpret_cast<float *>(smem_raw);                 // Npad x Kpad, canonical
  float *sX = sB + (size_t)Npad * Kpad;                             // S x 128 x KC, canonical
  __shared__ __align__(8) uint64_t mbar[S];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ncols_tmem)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    fail = 0;
    for (int i = 0; i < S; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // resident transform matrix, canonical layout with KG = Kpad / 4 core-matrix columns
  {
    const int KG = Kpad / 4;
    for (int idx = threadIdx.x; idx < Npad * Kpad; idx += blockDim.x) {
      int w = idx & 31, blk = idx >> 5;
      int rg = blk / KG, kg = blk - rg * KG;
      int r = rg * 8 + (w >> 2), k = kg * 4 + (w & 3);
      sB[idx] = Mp[(size_t)r * Kpad + k];
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = tf32_idesc(kTcRows, Npad);
  const uint32_t sboB = (uint32_t)(Kpad / 4) * 128, sboX = (kTcKC / 4) * 128;
  const int nchunks = Kpad / kTcKC;
  const long long ntiles = (R + kTcRows - 1) / kTcRows;
  const long long my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const long long njobs = my_tiles * nchunks;
  constexpr int KG = kTcKC / 4;

  auto issue = [&](long long q) {
    // cp.async of job q's X chunk into stage q % S (one commit group per job)
    if (q < njobs) {
      long long tile = blockIdx.x + (q / nchunks) * gridDim.x;
      int kc = (int)(q % nchunks) * kTcKC;
      long long row0 = tile * kTcRows;
      float *dst = sX + (size_t)(q % S) * kTcRows * kTcKC;
      for (int idx = threadIdx.x; idx < kTcRows * kTcKC; idx += blockDim.x) {
        int w = idx & 31, blk = idx >> 5;
        int rg = blk / KG, kg = blk - rg * KG;
        int r = rg * 8 + (w >> 2), k = kg * 4 + (w & 3);
        long long row = row0 + r;
        int kk = kc + k;
        bool ok = row < R && kk < nb;
        const float *src = ok ? X + row * nb + kk : X;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst + idx)), "l"(src),
                     "r"(ok ? 4 : 0)
                     : "memory");
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  for (int q = 0; q < S - 1; ++q) issue(q);
  for (long long q = 0; q < njobs; ++q) {
    // stage (q + S - 1) % S was last read by the MMAs of job q - 1
    if (q >= 1) {
      long long pq = q - 1;
      if (!mbar_wait(smem_u32(&mbar[pq % S]), (uint32_t)((pq / S) & 1), 1ll << 22)) fail = 1;
    }
    issue(q + S - 1);
    asm volatile("cp.async.wait_group %0;" ::"n"(S - 1) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (fail) break;
    const int chunk = (int)(q % nchunks);
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t xs = smem_u32(sX + (size_t)(q % S) * kTcRows * kTcKC);
#pragma unroll
      for (int s = 0; s < kTcKC / 8; ++s) {
        uint64_t ad = smem_desc(xs + 2 * s * 128, 128, sboX);
        uint64_t bd = smem_desc(smem_u32(sB) + (uint32_t)((chunk * KG + 2 * s) * 128), 128, sboB);
        uint32_t acc = (chunk > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar[q % S]))
                   : "memory");
    }
    if (chunk == nchunks - 1) {
      // tile complete: wait for its MMAs, then read the accumulator
      if (!mbar_wait(smem_u32(&mbar[q % S]), (uint32_t)((q / S) & 1), 1ll << 22)) fail = 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      __syncthreads();
      if (fail) break;
      const long long tile = blockIdx.x + (q / nchunks) * gridDim.x;
      const int lw = warp & 3, half = warp >> 2;
      const long long row = tile * kTcRows + lw * 32 + lane;
      long long t = 0, a = 0;
      if (row < R) {
        t = row / Aa;
        a = row - t * Aa;
      }
      for (int c0 = half * 16; c0 < Npad; c0 += 32) {
        uint32_t v[16];
        uint32_t taddr = tmem + ((uint32_t)(lw * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row < R) {
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            int j = c0 + u;
            if (j < nj) out[(t * nj + j) * Aa + a] = __uint_as_float(v[u]);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols_tmem) : "memory");
  }
  if (threadIdx.x == 0 && fail) atomicExch(err, 1);
}

}  // namespace

int tc_ncols(int npad) {
  int c = 32;
  while (c < npad) c <<= 1;
  return c;
}

// Launch one rotating transform on the tensor cores.  Requires nj <= 256.
st_status launch_tc_rot_gemm(cudaStream_t s, float *out, const float *X, const float *Mpad, long long R, int nb,
                             int nj, int Npad, int Kpad, long long Aa, int *err) {
  if (Npad > 256 || Npad % 16 != 0 || Kpad % kTcKC != 0) return ST_ERR_ARG;
  int ncols = tc_ncols(Npad);
  constexpr int S = 4;
  size_t need2 = ((size_t)Npad * Kpad + (size_t)S * kTcRows * kTcKC) * sizeof(float);
  if (need2 <= 200 * 1024) {
    static bool attr2 = false;
    if (!attr2) {
      ST_CUDA(cudaFuncSetAttribute(tc_rot_gemm2_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      attr2 = true;
    }
    long long ntiles2 = (R + kTcRows - 1) / kTcRows;
    int per_sm = std::max(1, std::min(512 / ncols, (int)((227 * 1024) / (need2 + 2048))));
    int grid2 = (int)std::min<long long>(ntiles2, 152LL * per_sm);
    st_count_launch();
    tc_rot_gemm2_kernel<S><<<grid2, 256, need2, s>>>(out, X, Mpad, R, nb, nj, Npad, Kpad, Aa, ncols, err);
    ST_CUDA(cudaGetLastError());
    return ST_OK;
  }
  size_t need = (size_t)(kTcRows + Npad) * kTcKC * sizeof(float);
  // limit resident CTAs per SM so that their tensor-memory columns fit in 512
  int max_ctas = 512 / ncols;
  size_t floor_bytes = (size_t)(227 * 1024) / (size_t)(max_ctas + 1) + 1024;
  size_t sh = std::max(need, floor_bytes);
  static bool attr_set = false;
  if (!attr_set) {
    ST_CUDA(cudaFuncSetAttribute(tc_rot_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  long long ntiles = (R + kTcRows - 1) / kTcRows;
  int grid = (int)std::min<long long>(ntiles, 152LL * max_ctas);
  st_count_launch();
  tc_rot_gemm_kernel<<<grid, 128, sh, s>>>(out, X, Mpad, R, nb, nj, Npad, Kpad, Aa, ncols, err);
  ST_CUDA(cudaGetLastError());
  return ST_OK;
}

namespace {
int g_tc_state = 0;
double g_tc_err = 0.0;

// host-side deterministic fill (linear congruential, values in [-1, 1))
void fill(std::vector<float> &v, unsigned seed) {
  unsigned x = seed;
  for (auto &e : v) {
    x = x * 1664525u + 1013904223u;
    e = (float)((x >> 8) * (1.0 / 8388608.0) - 1.0);
  }
}
}  // namespace

// One-time check of the tensor-core transform against the SIMT transform on
// a ragged problem (rows not a multiple of the tile, n not a multiple of 16).
int tc_state(cudaStream_t s, double *err_out) {
  if (g_tc_state != 0) {
    if (err_out) *err_out = g_tc_err;
    return g_tc_state;
  }
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10) {
    g_tc_state = -1;
    return g_tc_state;
  }
  const int nb = 131, nj = 131, T = 27;
  const long long Aa = 37, R = T * Aa;
  const int Npad = 144, Kpad = 160;
  std::vector<float> X((size_t)R * nb), M((size_t)nj * nb), Mp((size_t)Npad * Kpad, 0.0f);
  fill(X, 12345u);
  fill(M, 777u);
  for (int j = 0; j < nj; ++j)
    for (int k = 0; k < nb; ++k) Mp[(size_t)j * Kpad + k] = M[(size_t)j * nb + k];
  float *dX = nullptr, *dM = nullptr, *dMp = nullptr, *d1 = nullptr, *d2 = nullptr;
  int *derr = nullptr;
  size_t no = (size_t)T * nj * Aa;
  bool ok = cudaMalloc(&dX, X.size() * 4) == cudaSuccess && cudaMalloc(&dM, M.size() * 4) == cudaSuccess &&
            cudaMalloc(&dMp, Mp.size() * 4) == cudaSuccess && cudaMalloc(&d1, no * 4) == cudaSuccess &&
            cudaMalloc(&d2, no * 4) == cudaSuccess && cudaMalloc(&derr, 4) == cudaSuccess;
  double err = 1.0;
  if (ok) {
    cudaMemcpy(dX, X.data(), X.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(dM, M.data(), M.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(dMp, Mp.data(), Mp.size() * 4, cudaMemcpyHostToDevice);
    cudaMemset(derr, 0, 4);
    cudaMemset(d1, 0, no * 4);
    launch_rot_gemm<float>(s, d2, dX, dM, nb, nj, Aa, T);
    st_status st = launch_tc_rot_gemm(s, d1, dX, dMp, R, nb, nj, Npad, Kpad, Aa, derr);
    int herr = 1;
    if (st == ST_OK && cudaStreamSynchronize(s) == cudaSuccess) {
      cudaMemcpy(&herr, derr, 4, cudaMemcpyDeviceToHost);
      std::vector<float> o1(no), o2(no);
      cudaMemcpy(o1.data(), d1, no * 4, cudaMemcpyDeviceToHost);
      cudaMemcpy(o2.data(), d2, no * 4, cudaMemcpyDeviceToHost);
      double mx = 0.0, md = 0.0;
      for (size_t i = 0; i < no; ++i) {
        mx = std::max(mx, (double)std::fabs(o2[i]));
        double dd = std::fabs((double)o1[i] - (double)o2[i]);
        md = (dd == dd) ? std::max(md, dd) : 1e30;
      }
      err = mx > 0 ? md / mx : 1.0;
      if (herr) err = 1.0;
    }
    cudaGetLastError();
  }
  cudaFree(dX); cudaFree(dM); cudaFree(dMp); cudaFree(d1); cudaFree(d2); cudaFree(derr);
  g_tc_err = err;
  g_tc_state = (ok && err < 5e-3) ? 1 : -1;
  if (err_out) *err_out = err;
  return g_tc_state;
}
