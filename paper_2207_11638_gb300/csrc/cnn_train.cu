// Training of the CNN size selector: loss and gradient of a batch, and Adam.
//
// The network and its mixed precision are those of cnn.cuh.  A training
// step runs layer by layer over a batch of B regions (B a multiple of 64),
// every contraction a bfloat16 tensor-core GEMM with float32 accumulation:
//   forward   conv_l:  R_l = relu(im2col(a_{l-1}) W_l^T + b_l)  (bf16), pooled with its argmax
//             fc1:     u = h Wf1^T                               (float32)
//             head:    per slot logits, softmax, cross-entropy (+ expected
//                      normalised RD regret from the search's partition costs),
//                      d logits, d g, du = sum over slots (CUDA cores)
//   backward  fc1:     dh = du Wf1;  dWf1 = du^T h
//             conv_l:  dZ_l = scatter of d a_l to the window maxima, masked by R_l > 0 (bf16)
//                      dW_l = dZ_l^T im2col(a_{l-1});  db_l = column sums of dZ_l
//                      d a_{l-1} = im2col(dZ_l) W'_l^T with W'_l the tap-flipped,
//                      channel-transposed W_l (a 3 x 3 correlation's adjoint)
// Weight gradients are summed per chunk of rows into partial buffers, then
// reduced in a fixed order, so a step is reproducible bit for bit.
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "cnn.cuh"
#include "mma.cuh"
#include "common.cuh"
#include "ptx.cuh"
#include "tcgen05.cuh"

namespace cdct {
namespace {

using namespace cnn;

// ---------------------------------------------------------------------------
// GEMM  C[M][N] = A[M][K] B[N][K]^T on the tcgen05 tensor cores (bf16 in,
// float32 accumulate in tensor memory).  K % 16 == 0, N a multiple of BN
// (16, 32 or 64); rows of A beyond M read as zero.  A persistent CTA owns a
// column block of BN and walks the 128-row tiles t = blockIdx.x + i gridDim.x:
//   * B (BN x K) is copied into shared memory once, in the no-swizzle K-major
//     core-matrix layout: slab kk (K = 16) at kk * BN * 32 bytes, core matrices
//     128 B apart along K and 256 B apart along N;
//   * A arrives by TMA (cp.async.bulk.tensor through a tensor map of this GPU's
//     A[M][K]) in a ring of 4 stages of 64 K: one box of 8 K x 128 rows per
//     copy, so a stage holds chunk c of 8 K at c * 2048 + row * 16 bytes:
//     core matrices 2048 B apart along K and 128 B apart along M;
//   * one thread issues the copies (running up to 3 stages ahead) and the
//     MMAs, 4 per stage, into one of two tensor-memory accumulators;
//     tcgen05.commit frees a stage when its MMAs are done and publishes a tile
//     when its last MMA is;
//   * 4 epilogue warps drain a tile's accumulator (warp w: lanes 32w ..), hand
//     it back, and store: float32 out, or bias + ReLU -> bf16.
// So the copies of the next tiles, the MMAs of this one and the epilogue of
// the previous one overlap.  Every wait is bounded; a role that gives up
// raises a shared flag that ends the others' waits, the issuing thread waits
// (bounded) for its copies and MMAs in flight, and the CTA records the error
// word and frees its tensor memory.
// ---------------------------------------------------------------------------
constexpr int kGemmKS = 64;                        // K per pipeline stage
constexpr int kGemmStages = 4;
constexpr int kGemmStageBytes = 128 * kGemmKS * 2;
constexpr int kGemmEpiWarps = 4;
constexpr int kGemmThreads = 32 * (kGemmEpiWarps + 1);

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// wait for phase `parity`; false once the CTA has given up (the shared flag) or
// after about `limit` SM cycles, which also raises the flag
__device__ __forceinline__ bool gemm_wait(uint64_t* bar, uint32_t parity, long long limit, volatile int* abort) {
  if (mbar_try_wait(bar, parity, 2000u)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity, 2000u)) {
    if (*abort) return false;
    if (clock64() - t0 > limit) {
      *abort = 1;
      return false;
    }
  }
  return true;
}

// `skip_mma` (failure-detection test): issue neither the MMAs nor their
// commits, so that the waits run out with nothing but finished copies behind them.
template <int BN, bool RELU_BF16>
__global__ void __launch_bounds__(kGemmThreads, 1) gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                  const uint16_t* __restrict__ B, long long M, int N,
                                                                  int K, const float* __restrict__ bias,
                                                                  void* __restrict__ C, int* __restrict__ err,
                                                                  long long wait_limit, int skip_mma) {
  extern __shared__ __align__(1024) unsigned char smg[];
  __shared__ __align__(8) uint64_t full[kGemmStages], empty[kGemmStages], acc_full[2], acc_free[2], fin;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  volatile int* abort = &abort_flag;
  constexpr uint32_t kCols = 2 * BN < 32 ? 32 : 2 * BN;
  constexpr uint32_t kSlabB = BN * 32;             // bytes per K = 16 slab of B
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.y * BN;
  const int ks_per_tile = (K + kGemmKS - 1) / kGemmKS;
  const long long n_tiles = (M + 127) / 128;
  const long long my_tiles = (n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
  unsigned char* sb = smg;
  unsigned char* sa = smg + (BN * K * 2 + 1023) / 1024 * 1024;
  for (int i = tid; i < (K / 8) * BN; i += kGemmThreads) {
    const int kc = i / BN, r = i - kc * BN;
    *reinterpret_cast<uint4*>(sb + (kc >> 1) * kSlabB + (r >> 3) * 256 + (kc & 1) * 128 + (r & 7) * 16) =
        *reinterpret_cast<const uint4*>(B + static_cast<long long>(n0 + r) * K + kc * 8);
  }
  fence_proxy_async_smem();                // B is read by the tensor cores
  if (warp == 0) tmem_alloc(&tmem_base, kCols);
  if (tid == 0) {
    for (int j = 0; j < kGemmStages; ++j) {
      mbar_init(&full[j], 1);
      mbar_init(&empty[j], 1);
    }
    for (int j = 0; j < 2; ++j) {
      mbar_init(&acc_full[j], 1);
      mbar_init(&acc_free[j], kGemmEpiWarps);
    }
    mbar_init(&fin, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  if (warp == kGemmEpiWarps) {
    if (lane == 0) {
      // copies of stage g run kGemmStages - 1 stages ahead of the MMAs of stage g - (kGemmStages - 1)
      constexpr uint32_t idesc = idesc_bf16_f32(128, BN);
      const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
      const long long total = my_tiles * ks_per_tile;
      long long issued = 0;                        // stages whose copies were issued
      bool ok = true;
      for (long long g = 0; g < total + kGemmStages - 1; ++g) {
        if (g < total) {
          const int st = static_cast<int>(g % kGemmStages);
          const long long use = g / kGemmStages;
          if (use >= 1 && !gemm_wait(&empty[st], static_cast<uint32_t>((use - 1) & 1), wait_limit, abort)) {
            ok = false;
            break;
          }
          const long long tile = blockIdx.x + (g / ks_per_tile) * gridDim.x;
          const int k0 = static_cast<int>(g % ks_per_tile) * kGemmKS, kn = min(kGemmKS, K - k0);
          mbar_arrive_expect_tx(&full[st], static_cast<uint32_t>(kn / 8) * 2048u);
          for (int c = 0; c < kn / 8; ++c)
            tma_load_2d(sa + st * kGemmStageBytes + c * 2048, &tmA, k0 + 8 * c, static_cast<int>(tile * 128),
                        &full[st]);
          issued = g + 1;
        }
        const long long ci = g - (kGemmStages - 1);
        if (ci >= 0) {
          const int st = static_cast<int>(ci % kGemmStages);
          const long long ti = ci / ks_per_tile;
          const int s = static_cast<int>(ci % ks_per_tile), b = static_cast<int>(ti & 1);
          if (!gemm_wait(&full[st], static_cast<uint32_t>((ci / kGemmStages) & 1), wait_limit, abort) ||
              (s == 0 && ti >= 2 &&
               !gemm_wait(&acc_free[b], static_cast<uint32_t>(((ti - 2) >> 1) & 1), wait_limit, abort))) {
            ok = false;
            break;
          }
          tc_fence_after();
          if (!skip_mma) {
            const int k0 = s * kGemmKS, kn = min(kGemmKS, K - k0);
            for (int kk = 0; kk < kn / 16; ++kk)
              umma_bf16(tmem + b * BN, umma_desc(a0 + st * kGemmStageBytes + 2 * kk * 2048, 2048, 128),
                        umma_desc(b0 + (k0 / 16 + kk) * kSlabB, 128, 256), idesc, (s > 0 || kk > 0) ? 1u : 0u);
            umma_commit(&empty[st]);
            if (s == ks_per_tile - 1) umma_commit(&acc_full[b]);
          }
        }
      }
      if (!ok) *abort = 1;
      // nothing may still write this CTA's memory when it exits: the MMAs issued
      // (one commit tracks them all) and the copies issued (each stage's last)
      umma_commit(&fin);
      (void)mbar_wait_bounded(&fin, 0u, wait_limit);
      for (long long g = issued - 1; g >= 0 && g >= issued - kGemmStages; --g)
        (void)mbar_wait_bounded(&full[g % kGemmStages], static_cast<uint32_t>((g / kGemmStages) & 1), wait_limit);
    }
    __syncwarp();
  } else {
    for (long long ti = 0; ti < my_tiles; ++ti) {
      const int b = static_cast<int>(ti & 1);
      const bool ok = __all_sync(0xffffffffu, gemm_wait(&acc_full[b], static_cast<uint32_t>((ti >> 1) & 1),
                                                        wait_limit, abort));
      if (!ok) break;
      tc_fence_after();
      float v[BN];
#pragma unroll
      for (int c0 = 0; c0 < BN; c0 += 16)
        tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + b * BN + c0,
                  *reinterpret_cast<float(*)[16]>(v + c0));
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_free[b]);   // the accumulator is free for tile ti + 2
      const long long row = (blockIdx.x + ti * gridDim.x) * 128 + warp * 32 + lane;
      if (row < M) {
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
          const int col = n0 + c0;
          if (RELU_BF16) {
            uint32_t w[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
              w[j] = pack_bf16(fmaxf(v[c0 + 2 * j] + bias[col + 2 * j], 0.f),
                               fmaxf(v[c0 + 2 * j + 1] + bias[col + 2 * j + 1], 0.f));
            uint4* dst = reinterpret_cast<uint4*>(static_cast<uint16_t*>(C) + row * N + col);
            dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
            dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
          } else {
            float4* dst = reinterpret_cast<float4*>(static_cast<float*>(C) + row * N + col);
#pragma unroll
            for (int j = 0; j < 4; ++j)
              dst[j] = make_float4(v[c0 + 4 * j], v[c0 + 4 * j + 1], v[c0 + 4 * j + 2], v[c0 + 4 * j + 3]);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && abort_flag) atomicOr(err, 2);
  if (warp == 0) tmem_dealloc(tmem, kCols);
}

// cuTensorMapEncodeTiled, fetched from the driver once (no link-time dependency on it)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// SMs of the current device, looked up once per device (safe to call from several host threads)
int sm_count() {
  static std::atomic<int> n[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  int v = n[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    n[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

template <int BN, bool RELU_BF16>
int gemm_launch_t(const uint16_t* A, const uint16_t* B, long long M, int N, int K, const float* bias, void* C,
                  int* err, cudaStream_t s) {
  EncodeTiledFn enc = encode_tiled();
  const int sms = sm_count();
  if (enc == nullptr || sms <= 0) return static_cast<int>(cudaErrorNotSupported);
  CUtensorMap map;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(K), static_cast<cuuint64_t>(M)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(K) * 2};
  const cuuint32_t box[2] = {8, 128};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t*>(A), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return static_cast<int>(cudaErrorInvalidValue);
  const int smem = (BN * K * 2 + 1023) / 1024 * 1024 + kGemmStages * kGemmStageBytes;
  auto kern = gemm_tc_kernel<BN, RELU_BF16>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return static_cast<int>(e);
  const long long tiles = (M + 127) / 128;
  const int cols = N / BN;
  const long long want = (sms + cols - 1) / cols;   // about one CTA per SM over the column blocks
  dim3 grid(static_cast<unsigned>(tiles < want ? tiles : want), static_cast<unsigned>(cols));
  long long limit = kDefaultWaitLimit;
  const int mode = fault_mode(&limit);
  kern<<<grid, kGemmThreads, smem, s>>>(map, B, M, N, K, bias, C, err, limit, (mode & 2) ? 1 : 0);
  return static_cast<int>(cudaGetLastError());
}

int gemm(const uint16_t* A, const uint16_t* B, long long M, int N, int K, const float* bias, void* C, bool relu_bf16,
         int* err, cudaStream_t s) {
  if (N == 16) return relu_bf16 ? gemm_launch_t<16, true>(A, B, M, N, K, bias, C, err, s)
                                : gemm_launch_t<16, false>(A, B, M, N, K, bias, C, err, s);
  if (N == 32) return relu_bf16 ? gemm_launch_t<32, true>(A, B, M, N, K, bias, C, err, s)
                                : gemm_launch_t<32, false>(A, B, M, N, K, bias, C, err, s);
  return relu_bf16 ? gemm_launch_t<64, true>(A, B, M, N, K, bias, C, err, s)
                   : gemm_launch_t<64, false>(A, B, M, N, K, bias, C, err, s);
}

// ---------------------------------------------------------------------------
// Weight gradient  P[chunk][Co][K] = sum over the chunk's rows m of dZ[m][co] A[m][k]
// (and Pb[chunk][co] = sum of dZ[m][co]).  Chunks of MCH rows; a CTA of 4
// warps owns 64 columns of A, a warp 16 of them (two n-tiles) for every
// 16-row tile of co.  Both operands are read transposed with ldmatrix.trans
// from row-major tiles in shared memory.
// ---------------------------------------------------------------------------
template <int CO>
__global__ void __launch_bounds__(128) wgrad_kernel(const uint16_t* __restrict__ dZ, const uint16_t* __restrict__ A,
                                                    int K, int mch, float* __restrict__ part,
                                                    float* __restrict__ part_b) {
  extern __shared__ __align__(16) unsigned char smw[];
  constexpr int zp = CO + 8;
  constexpr int ap = 64 + 8;
  uint16_t* sz = reinterpret_cast<uint16_t*>(smw);
  uint16_t* sa = sz + mch * zp;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long r0 = static_cast<long long>(blockIdx.x) * mch;
  const int c0 = blockIdx.y * 64;
  const int cols = min(64, K - c0);
  for (int i = tid; i < mch * (CO / 8); i += 128) {
    const int r = i / (CO / 8), c = i - r * (CO / 8);
    *reinterpret_cast<uint4*>(sz + r * zp + c * 8) = *reinterpret_cast<const uint4*>(dZ + (r0 + r) * CO + c * 8);
  }
  for (int i = tid; i < mch * 8; i += 128) {
    const int r = i >> 3, c = i & 7;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (c * 8 < cols) v = *reinterpret_cast<const uint4*>(A + (r0 + r) * K + c0 + c * 8);
    *reinterpret_cast<uint4*>(sa + r * ap + c * 8) = v;
  }
  __syncthreads();
  if (blockIdx.y == 0 && tid < CO) {
    float s = 0.f;
    for (int r = 0; r < mch; ++r) s += __uint_as_float(static_cast<uint32_t>(sz[r * zp + tid]) << 16);
    part_b[blockIdx.x * CO + tid] = s;
  }
  if (warp * 16 >= cols) return;
  float acc[CO / 16][2][4];
#pragma unroll
  for (int i = 0; i < CO / 16; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
  const int j = lane >> 3;
  // A_mma[co][m] from sz[m][co]: matrix j = (m half j >> 1, co half j & 1)
  const uint32_t z_lane = smem_u32(sz) + (((j >> 1) * 8 + (lane & 7)) * zp + (j & 1) * 8) * 2;
  // B_mma[m][k] from sa[m][k]: matrix j = (m half j & 1, k half j >> 1)
  const uint32_t a_lane = smem_u32(sa) + (((j & 1) * 8 + (lane & 7)) * ap + warp * 16 + (j >> 1) * 8) * 2;
  for (int m = 0; m < mch; m += 16) {
    uint32_t bf[4];
    ldsm_x4_t(bf, a_lane + m * ap * 2);
    const uint32_t b0[2] = {bf[0], bf[1]}, b1[2] = {bf[2], bf[3]};
#pragma unroll
    for (int ct = 0; ct < CO / 16; ++ct) {
      uint32_t af[4];
      ldsm_x4_t(af, z_lane + (m * zp + ct * 16) * 2);
      mma_bf16(acc[ct][0], af, b0);
      mma_bf16(acc[ct][1], af, b1);
    }
  }
  const int g = lane >> 2, t = lane & 3;
  float* out = part + static_cast<long long>(blockIdx.x) * CO * K;
#pragma unroll
  for (int ct = 0; ct < CO / 16; ++ct)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const int col = c0 + warp * 16 + nt * 8 + 2 * t;
      if (col < K) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int co = ct * 16 + g + 8 * h;
          *reinterpret_cast<float2*>(out + co * K + col) = make_float2(acc[ct][nt][2 * h], acc[ct][nt][2 * h + 1]);
        }
      }
    }
}

// out[co * kreal + k] = sum over chunks of part[chunk][co][k] for k < kreal; bias likewise.
// A CTA of 32 warps owns 32 consecutive outputs (lane = output, so loads are
// coalesced along k); warp w sums chunks w, w + 32, w + 64, ... in that order,
// then warp 0 adds the 32 warps' sums in warp order: a fixed order, so the
// result is the same bit for bit on every run.
constexpr int kReduceWarps = 32;
__global__ void __launch_bounds__(32 * kReduceWarps) wgrad_reduce_kernel(const float* __restrict__ part,
                                                                         const float* __restrict__ part_b, int chunks,
                                                                         int co_n, int K, int kreal,
                                                                         float* __restrict__ gw, float* __restrict__ gb) {
  __shared__ float red[kReduceWarps][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_w = co_n * kreal, n_out = n_w + (gb != nullptr ? co_n : 0);
  const int e = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (e < n_w) {
    const int co = e / kreal, k = e - co * kreal;
    const float* p = part + static_cast<long long>(co) * K + k;
    const long long step = static_cast<long long>(co_n) * K;
#pragma unroll 4
    for (int c = warp; c < chunks; c += kReduceWarps) s += p[c * step];
  } else if (e < n_out) {
    const int co = e - n_w;
#pragma unroll 4
    for (int c = warp; c < chunks; c += kReduceWarps) s += part_b[c * co_n + co];
  }
  red[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && e < n_out) {
    float t = red[0][lane];
    for (int w = 1; w < kReduceWarps; ++w) t += red[w][lane];
    if (e < n_w) gw[e] = t;
    else gb[e - n_w] = t;
  }
}

template <int CO>
int wgrad_launch_t(const uint16_t* dZ, const uint16_t* A, long long M, int K, int kreal, float* part, float* part_b,
                   float* gw, float* gb, cudaStream_t s) {
  const int mch = (M % 256 == 0) ? 256 : 64;
  const int smem = mch * (CO + 8) * 2 + mch * 72 * 2;
  auto kern = wgrad_kernel<CO>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return static_cast<int>(e);
  const int chunks = static_cast<int>(M / mch);
  dim3 grid(chunks, (K + 63) / 64);
  kern<<<grid, 128, smem, s>>>(dZ, A, K, mch, part, part_b);
  e = cudaGetLastError();
  if (e != cudaSuccess) return static_cast<int>(e);
  const int total = CO * kreal + (gb ? CO : 0);
  wgrad_reduce_kernel<<<(total + 31) / 32, 32 * kReduceWarps, 0, s>>>(part, part_b, chunks, CO, K, kreal, gw, gb);
  return static_cast<int>(cudaGetLastError());
}

int wgrad(int co, const uint16_t* dZ, const uint16_t* A, long long M, int K, int kreal, float* part, float* part_b,
          float* gw, float* gb, cudaStream_t s) {
  if (co == 16) return wgrad_launch_t<16>(dZ, A, M, K, kreal, part, part_b, gw, gb, s);
  if (co == 32) return wgrad_launch_t<32>(dZ, A, M, K, kreal, part, part_b, gw, gb, s);
  return wgrad_launch_t<64>(dZ, A, M, K, kreal, part, part_b, gw, gb, s);
}

// ---------------------------------------------------------------------------
// im2col of a 3 x 3, zero-padded correlation: A[(b, y, x)][tap * C + c] = X[b][y + dy - 1][x + dx - 1][c]
// ---------------------------------------------------------------------------
template <int C>
__global__ void im2col_kernel(const uint16_t* __restrict__ X, int H, long long total, uint16_t* __restrict__ A) {
  constexpr int V = C / 8;   // uint4 per pixel
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int v = static_cast<int>(i % V);
    const long long q = i / V;
    const int tap = static_cast<int>(q % 9);
    const long long m = q / 9;
    const int x = static_cast<int>(m % H), y = static_cast<int>((m / H) % H);
    const long long b = m / (static_cast<long long>(H) * H);
    const int sy = y + tap / 3 - 1, sx = x + tap % 3 - 1;
    uint4 val = make_uint4(0, 0, 0, 0);
    if (sy >= 0 && sy < H && sx >= 0 && sx < H)
      val = *reinterpret_cast<const uint4*>(X + ((b * H + sy) * H + sx) * C + v * 8);
    *reinterpret_cast<uint4*>(A + m * (9 * C) + tap * C + v * 8) = val;
  }
}

// layer-1 im2col straight from the int16 regions: A[(b, y, x)][k] = bf16(x[...] / 64) for k < 9, 0 for k = 9..15
__global__ void im2col_input_kernel(const int16_t* __restrict__ X, long long total, uint16_t* __restrict__ A) {
  for (long long m = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; m < total;
       m += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int x = static_cast<int>(m & 31), y = static_cast<int>((m >> 5) & 31);
    const long long b = m >> 10;
    uint32_t w[8];
#pragma unroll
    for (int k = 0; k < 16; k += 2) {
      uint32_t lo = 0, hi = 0;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int kk = k + e;
        uint32_t bits = 0;
        if (kk < 9) {
          const int sy = y + kk / 3 - 1, sx = x + kk % 3 - 1;
          if (sy >= 0 && sy < 32 && sx >= 0 && sx < 32)
            bits = bf16_bits(static_cast<float>(X[(b * 32 + sy) * 32 + sx]) * 0.015625f);
        }
        if (e == 0) lo = bits; else hi = bits;
      }
      w[k / 2] = lo | (hi << 16);
    }
    uint4* dst = reinterpret_cast<uint4*>(A + m * 16);
    dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
    dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
  }
}

// ---------------------------------------------------------------------------
// 2 x 2 max pool (first maximum in raster order) and its adjoint
// ---------------------------------------------------------------------------
__global__ void pool_kernel(const uint16_t* __restrict__ R, int H, int C, long long total, uint16_t* __restrict__ P,
                            uint8_t* __restrict__ arg) {
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(i % C);
    const long long q = i / C;
    const int h2 = H / 2;
    const int px = static_cast<int>(q % h2), py = static_cast<int>((q / h2) % h2);
    const long long b = q / (static_cast<long long>(h2) * h2);
    uint16_t best = 0;
    float bv = -1.f;
    int ba = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint16_t v = R[((b * H + 2 * py + (k >> 1)) * H + 2 * px + (k & 1)) * C + c];
      const float f = __uint_as_float(static_cast<uint32_t>(v) << 16);
      if (f > bv) { bv = f; best = v; ba = k; }
    }
    P[i] = best;
    arg[i] = static_cast<uint8_t>(ba);
  }
}

// dZ[b][y][x][c] = bf16(dP[b][y/2][x/2][c]) where (y, x) is the window's maximum and R > 0, else 0
__global__ void pool_backward_kernel(const float* __restrict__ dP, const uint8_t* __restrict__ arg,
                                     const uint16_t* __restrict__ R, int H, int C, long long total,
                                     uint16_t* __restrict__ dZ) {
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(i % C);
    const long long q = i / C;
    const int x = static_cast<int>(q % H), y = static_cast<int>((q / H) % H);
    const long long b = q / (static_cast<long long>(H) * H);
    const int h2 = H / 2;
    const long long pi = ((b * h2 + y / 2) * h2 + x / 2) * C + c;
    uint16_t out = 0;
    if (arg[pi] == ((y & 1) * 2 + (x & 1)) && R[i] != 0) out = bf16_bits(dP[pi]);
    dZ[i] = out;
  }
}

// ---------------------------------------------------------------------------
// bf16 weight copies for the GEMMs: forward W_l [Co][K] (conv1 zero-padded to
// K = 16), tap-flipped transposes W'_l [Ci][9 Co] for the input gradients,
// Wf1 [64][512] and Wf1^T [512][64].
// ---------------------------------------------------------------------------
struct PrepOut {
  uint16_t *w1, *w2, *w3, *w2f, *w3f, *f1, *f1t;
};

__global__ void prep_weights_kernel(const float* __restrict__ p, PrepOut o) {
  constexpr int n1 = 16 * 16, n2 = 32 * 144, n3 = 32 * 288, n2f = 16 * 288, n3f = 32 * 288, nf = 64 * 512;
  constexpr int total = n1 + n2 + n3 + n2f + n3f + nf + nf;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int k = i;
    if (k < n1) { const int co = k / 16, c = k % 16; o.w1[k] = bf16_bits(c < 9 ? p[kOffW1 + co * 9 + c] : 0.f); continue; }
    k -= n1;
    if (k < n2) { o.w2[k] = bf16_bits(p[kOffW2 + k]); continue; }
    k -= n2;
    if (k < n3) { o.w3[k] = bf16_bits(p[kOffW3 + k]); continue; }
    k -= n3;
    if (k < n2f) {   // W'2[ci][tap * 32 + co] = W2[co][8 - tap][ci]
      const int ci = k / 288, r = k % 288, tap = r / 32, co = r % 32;
      o.w2f[k] = bf16_bits(p[kOffW2 + (co * 9 + 8 - tap) * 16 + ci]);
      continue;
    }
    k -= n2f;
    if (k < n3f) {
      const int ci = k / 288, r = k % 288, tap = r / 32, co = r % 32;
      o.w3f[k] = bf16_bits(p[kOffW3 + (co * 9 + 8 - tap) * 32 + ci]);
      continue;
    }
    k -= n3f;
    if (k < nf) { o.f1[k] = bf16_bits(p[kOffF1 + k]); continue; }
    k -= nf;
    { const int f = k / 64, h = k % 64; o.f1t[k] = bf16_bits(p[kOffF1 + h * kFeat + f]); }
  }
}

// ---------------------------------------------------------------------------
// Head: per region (one warp) and slot, logits, softmax cross-entropy plus
// mu x expected normalised regret, and the gradients below the logits.
// A CTA of 8 warps covers 32 regions and writes one partial of
// [dWf2 (17 x 64) | dbf2 (17) | dWq (64 x 4) | dbf1 (64) | loss (1)].
// ---------------------------------------------------------------------------
constexpr int kHeadPart = kLabels * kHidden + kLabels + kHidden * kSlots + kHidden + 1;
constexpr int kHeadRegionsPerCta = 32;

struct HeadArgs {
  const float* p;          // params
  const float* u;          // [B][64]
  const uint8_t* labels;   // [ns][B]
  const unsigned long long* pcost;   // [ns][B][17][2] partition costs J' (low, high words) or null
  float mu, inv_count;
  int B, ns;
  int slots[kSlots];
  uint16_t* du;            // [B][64] bf16
  float* part;             // [B / 32][kHeadPart]
};

__global__ void __launch_bounds__(256) head_kernel(const HeadArgs a) {
  __shared__ float s_w2[kLabels * kHidden];
  __shared__ float s_q[kHidden * kSlots];
  __shared__ float s_b1[kHidden], s_b2[kLabels];
  __shared__ float s_g[8][kHidden];
  __shared__ float s_dl[8][kLabels + 1];
  __shared__ float s_acc[kHeadPart];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < kLabels * kHidden; i += 256) s_w2[i] = round_bf16(a.p[kOffF2 + i]);
  for (int i = tid; i < kHidden * kSlots; i += 256) s_q[i] = round_bf16(a.p[kOffQ + i]);
  for (int i = tid; i < kHeadPart; i += 256) s_acc[i] = 0.f;
  if (tid < kHidden) s_b1[tid] = a.p[kOffFB1 + tid];
  if (tid < kLabels) s_b2[tid] = a.p[kOffFB2 + tid];
  __syncthreads();
  // per-lane partials: hidden units h = lane, lane + 32; labels j = lane (< 17)
  float p2[kLabels][2], pq[kSlots][2], pb1[2] = {0.f, 0.f}, pb2 = 0.f, ploss = 0.f;
#pragma unroll
  for (int j = 0; j < kLabels; ++j) p2[j][0] = p2[j][1] = 0.f;
#pragma unroll
  for (int k = 0; k < kSlots; ++k) pq[k][0] = pq[k][1] = 0.f;
  for (int rr = 0; rr < kHeadRegionsPerCta / 8; ++rr) {
    const int region = blockIdx.x * kHeadRegionsPerCta + rr * 8 + warp;
    const float* ur = a.u + static_cast<long long>(region) * kHidden;
    const float u0 = ur[lane], u1 = ur[lane + 32];
    float du0 = 0.f, du1 = 0.f;
#pragma unroll
    for (int si = 0; si < kSlots; ++si) {
      if (si >= a.ns) break;
      const int slot = a.slots[si];
      const float g0 = round_bf16(fmaxf((u0 + s_b1[lane]) + s_q[lane * kSlots + slot], 0.f));
      const float g1 = round_bf16(fmaxf((u1 + s_b1[lane + 32]) + s_q[(lane + 32) * kSlots + slot], 0.f));
      s_g[warp][lane] = g0;
      s_g[warp][lane + 32] = g1;
      __syncwarp();
      float logit = -INFINITY;
      if (lane < kLabels) {
        float acc = s_b2[lane];
        for (int h = 0; h < kHidden; ++h) acc = fmaf(s_w2[lane * kHidden + h], s_g[warp][h], acc);
        logit = acc;
      }
      float mx = logit;
      for (int o = 16; o >= 1; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const float e = lane < kLabels ? expf(logit - mx) : 0.f;
      float se = e;
      for (int o = 16; o >= 1; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
      const float pj = e / se;
      int label = a.labels[static_cast<long long>(si) * a.B + region];
      label = label < kLabels ? label : kLabels - 1;
      const float plab = __shfl_sync(0xffffffffu, pj, label);
      float dl = pj - (lane == label ? 1.f : 0.f);
      float lossv = -logf(plab);
      if (a.pcost != nullptr && a.mu != 0.f) {
        // normalised regret c_j = (J_j - J_min) / J_min of the search's 17 partition costs
        double jv = INFINITY;
        if (lane < kLabels) {
          const unsigned long long* w = a.pcost + ((static_cast<long long>(si) * a.B + region) * kLabels + lane) * 2;
          jv = static_cast<double>(w[1]) * 18446744073709551616.0 + static_cast<double>(w[0]);
        }
        double jmin = jv;
        for (int o = 16; o >= 1; o >>= 1) jmin = fmin(jmin, __shfl_xor_sync(0xffffffffu, jmin, o));
        const float c = (lane < kLabels && jmin > 0.0) ? static_cast<float>((jv - jmin) / jmin) : 0.f;
        float er = pj * c;
        for (int o = 16; o >= 1; o >>= 1) er += __shfl_xor_sync(0xffffffffu, er, o);
        dl += a.mu * pj * (c - er);
        lossv += a.mu * er;
      }
      dl = lane < kLabels ? dl * a.inv_count : 0.f;
      if (lane < kLabels) s_dl[warp][lane] = dl;
      ploss += lossv;
      pb2 += dl;
      __syncwarp();
      // dg = Wf2^T dl masked by g > 0; dWf2 += dl g^T
      float dg0 = 0.f, dg1 = 0.f;
#pragma unroll
      for (int j = 0; j < kLabels; ++j) {
        const float d = s_dl[warp][j];
        dg0 = fmaf(s_w2[j * kHidden + lane], d, dg0);
        dg1 = fmaf(s_w2[j * kHidden + lane + 32], d, dg1);
        p2[j][0] = fmaf(d, g0, p2[j][0]);
        p2[j][1] = fmaf(d, g1, p2[j][1]);
      }
      dg0 = g0 > 0.f ? dg0 : 0.f;
      dg1 = g1 > 0.f ? dg1 : 0.f;
      pq[si][0] += dg0;
      pq[si][1] += dg1;
      pb1[0] += dg0;
      pb1[1] += dg1;
      du0 += dg0;
      du1 += dg1;
      __syncwarp();
    }
    a.du[static_cast<long long>(region) * kHidden + lane] = bf16_bits(du0);
    a.du[static_cast<long long>(region) * kHidden + lane + 32] = bf16_bits(du1);
  }
  // warps add their partials into s_acc one after another (fixed order)
  float* sq = s_acc + kLabels * kHidden + kLabels;
  for (int w = 0; w < 8; ++w) {
    if (warp == w) {
#pragma unroll
      for (int j = 0; j < kLabels; ++j) {
        s_acc[j * kHidden + lane] += p2[j][0];
        s_acc[j * kHidden + lane + 32] += p2[j][1];
      }
      if (lane < kLabels) s_acc[kLabels * kHidden + lane] += pb2;
#pragma unroll
      for (int si = 0; si < kSlots; ++si) {
        if (si < a.ns) {
          sq[lane * kSlots + a.slots[si]] += pq[si][0];
          sq[(lane + 32) * kSlots + a.slots[si]] += pq[si][1];
        }
      }
      s_acc[kLabels * kHidden + kLabels + kHidden * kSlots + lane] += pb1[0];
      s_acc[kLabels * kHidden + kLabels + kHidden * kSlots + lane + 32] += pb1[1];
      if (lane == 0) s_acc[kHeadPart - 1] += ploss;
    }
    __syncthreads();
  }
  for (int i = tid; i < kHeadPart; i += 256) a.part[static_cast<long long>(blockIdx.x) * kHeadPart + i] = s_acc[i];
}

// grad of the head parameters and the loss, summed over the CTA partials in order
__global__ void head_reduce_kernel(const float* __restrict__ part, int nparts, float* __restrict__ grad,
                                   float* __restrict__ loss, float inv_count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kHeadPart) return;
  float s = 0.f;
  for (int c = 0; c < nparts; ++c) s += part[static_cast<long long>(c) * kHeadPart + i];
  constexpr int a = kLabels * kHidden, b = a + kLabels, c = b + kHidden * kSlots, d = c + kHidden;
  if (i < a) grad[kOffF2 + i] = s;
  else if (i < b) grad[kOffFB2 + i - a] = s;
  else if (i < c) grad[kOffQ + i - b] = s;
  else if (i < d) grad[kOffFB1 + i - c] = s;
  else *loss = s * inv_count;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ---------------------------------------------------------------------------
// workspace carving
// ---------------------------------------------------------------------------
struct TrainWs {
  uint16_t *w1, *w2, *w3, *w2f, *w3f, *f1, *f1t;
  uint16_t *A1, *R1, *P1, *A2, *R2, *P2, *A3, *R3, *H;
  uint8_t *arg1, *arg2, *arg3;
  float* U;
  uint16_t* DU;
  float* DH;
  uint16_t *DZ3, *DZ2, *DZ1, *IMD;
  float *DA2, *DA1;
  float *wpart, *bpart, *hpart;
  size_t bytes;
};

TrainWs carve(void* base, long long B) {
  TrainWs w;
  unsigned char* p = static_cast<unsigned char*>(base);
  size_t off = 0;
  auto take = [&](size_t n) {
    unsigned char* r = p ? p + off : nullptr;
    off += (n + 255) / 256 * 256;
    return r;
  };
  auto bf = [&](size_t n) { return reinterpret_cast<uint16_t*>(take(n * 2)); };
  auto f32 = [&](size_t n) { return reinterpret_cast<float*>(take(n * 4)); };
  w.w1 = bf(16 * 16); w.w2 = bf(32 * 144); w.w3 = bf(32 * 288); w.w2f = bf(16 * 288); w.w3f = bf(32 * 288);
  w.f1 = bf(64 * 512); w.f1t = bf(512 * 64);
  w.A1 = bf(B * 1024 * 16); w.R1 = bf(B * 1024 * 16); w.P1 = bf(B * 256 * 16);
  w.A2 = bf(B * 256 * 144); w.R2 = bf(B * 256 * 32); w.P2 = bf(B * 64 * 32);
  w.A3 = bf(B * 64 * 288); w.R3 = bf(B * 64 * 32); w.H = bf(B * 512);
  w.arg1 = take(B * 256 * 16); w.arg2 = take(B * 64 * 32); w.arg3 = take(B * 512);
  w.U = f32(B * 64); w.DU = bf(B * 64); w.DH = f32(B * 512);
  w.DZ3 = bf(B * 64 * 32); w.DZ2 = bf(B * 256 * 32); w.DZ1 = bf(B * 1024 * 16);
  w.IMD = bf(B * 256 * 288);
  w.DA2 = f32(B * 64 * 32); w.DA1 = f32(B * 256 * 16);
  // weight-gradient partials: the largest of conv1 (B*1024/256 chunks x 16 x 16),
  // conv2 (B*256/256 x 32 x 144), conv3 (B*64/256 x 32 x 288), fc1 (B/64 x 64 x 512)
  long long wp = B * 4 * 16 * 16;
  wp = wp > B * 32 * 144 ? wp : B * 32 * 144;
  wp = wp > B / 4 * 32 * 288 ? wp : B / 4 * 32 * 288;
  wp = wp > B / 64 * 64 * 512 ? wp : B / 64 * 64 * 512;
  w.wpart = f32(wp);
  w.bpart = f32(B * 4 * 64);
  w.hpart = f32(B / kHeadRegionsPerCta * kHeadPart);
  w.bytes = off;
  return w;
}

int grid_for(long long n, int threads = 256) {
  long long g = (n + threads - 1) / threads;
  return static_cast<int>(g < 4096 ? g : 4096);
}

}  // namespace

size_t cnn_train_workspace(long long batch) { return carve(nullptr, batch).bytes; }

// Loss and gradient of one batch (see the file comment).  Returns a cudaError_t code.
int cnn_grad_launch(const float* params, const int16_t* regions, int B, const int* slots, int ns,
                    const unsigned char* labels, const unsigned long long* pcost, float mu, float* grad,
                    float* loss, void* workspace, int* err, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TrainWs w = carve(workspace, B);
  const long long b = B;
  int rc;
#define CNN_CHECK(x) do { rc = (x); if (rc) return rc; } while (0)
#define CNN_LAUNCHED() do { rc = static_cast<int>(cudaGetLastError()); if (rc) return rc; } while (0)
  prep_weights_kernel<<<128, 256, 0, s>>>(params, PrepOut{w.w1, w.w2, w.w3, w.w2f, w.w3f, w.f1, w.f1t});
  CNN_LAUNCHED();
  // forward
  im2col_input_kernel<<<grid_for(b * 1024), 256, 0, s>>>(regions, b * 1024, w.A1);
  CNN_LAUNCHED();
  CNN_CHECK(gemm(w.A1, w.w1, b * 1024, 16, 16, params + kOffB1, w.R1, true, err, s));
  pool_kernel<<<grid_for(b * 256 * 16), 256, 0, s>>>(w.R1, 32, 16, b * 256 * 16, w.P1, w.arg1);
  CNN_LAUNCHED();
  im2col_kernel<16><<<grid_for(b * 256 * 9 * 2), 256, 0, s>>>(w.P1, 16, b * 256 * 9 * 2, w.A2);
  CNN_LAUNCHED();
  CNN_CHECK(gemm(w.A2, w.w2, b * 256, 32, 144, params + kOffB2, w.R2, true, err, s));
  pool_kernel<<<grid_for(b * 64 * 32), 256, 0, s>>>(w.R2, 16, 32, b * 64 * 32, w.P2, w.arg2);
  CNN_LAUNCHED();
  im2col_kernel<32><<<grid_for(b * 64 * 9 * 4), 256, 0, s>>>(w.P2, 8, b * 64 * 9 * 4, w.A3);
  CNN_LAUNCHED();
  CNN_CHECK(gemm(w.A3, w.w3, b * 64, 32, 288, params + kOffB3, w.R3, true, err, s));
  pool_kernel<<<grid_for(b * 512), 256, 0, s>>>(w.R3, 8, 32, b * 512, w.H, w.arg3);
  CNN_LAUNCHED();
  CNN_CHECK(gemm(w.H, w.f1, b, 64, 512, nullptr, w.U, false, err, s));
  // head
  HeadArgs ha;
  ha.p = params;
  ha.u = w.U;
  ha.labels = labels;
  ha.pcost = pcost;
  ha.mu = mu;
  ha.inv_count = 1.f / static_cast<float>(b * ns);
  ha.B = B;
  ha.ns = ns;
  for (int k = 0; k < kSlots; ++k) ha.slots[k] = k < ns ? slots[k] : 0;
  ha.du = w.DU;
  ha.part = w.hpart;
  head_kernel<<<B / kHeadRegionsPerCta, 256, 0, s>>>(ha);
  CNN_LAUNCHED();
  head_reduce_kernel<<<(kHeadPart + 255) / 256, 256, 0, s>>>(w.hpart, B / kHeadRegionsPerCta, grad, loss,
                                                              ha.inv_count);
  CNN_LAUNCHED();
  // fc1 backward
  CNN_CHECK(gemm(w.DU, w.f1t, b, 512, 64, nullptr, w.DH, false, err, s));
  CNN_CHECK(wgrad(64, w.DU, w.H, b, 512, 512, w.wpart, w.bpart, grad + kOffF1, nullptr, s));
  // conv3
  pool_backward_kernel<<<grid_for(b * 64 * 32), 256, 0, s>>>(w.DH, w.arg3, w.R3, 8, 32, b * 64 * 32, w.DZ3);
  CNN_LAUNCHED();
  CNN_CHECK(wgrad(32, w.DZ3, w.A3, b * 64, 288, 288, w.wpart, w.bpart, grad + kOffW3, grad + kOffB3, s));
  im2col_kernel<32><<<grid_for(b * 64 * 9 * 4), 256, 0, s>>>(w.DZ3, 8, b * 64 * 9 * 4, w.IMD);
  CNN_LAUNCHED();
  CNN_CHECK(gemm(w.IMD, w.w3f, b * 64, 32, 288, nullptr, w.DA2, false, err, s));
  // conv2
  pool_backward_kernel<<<grid_for(b * 256 * 32), 256, 0, s>>>(w.DA2, w.arg2, w.R2, 16, 32, b * 256 * 32, w.DZ2);
  CNN_LAUNCHED();
  CNN_CHECK(wgrad(32, w.DZ2, w.A2, b * 256, 144, 144, w.wpart, w.bpart, grad + kOffW2, grad + kOffB2, s));
  im2col_kernel<32><<<grid_for(b * 256 * 9 * 4), 256, 0, s>>>(w.DZ2, 16, b * 256 * 9 * 4, w.IMD);
  CNN_LAUNCHED();
  CNN_CHECK(gemm(w.IMD, w.w2f, b * 256, 16, 288, nullptr, w.DA1, false, err, s));
  // conv1
  pool_backward_kernel<<<grid_for(b * 1024 * 16), 256, 0, s>>>(w.DA1, w.arg1, w.R1, 32, 16, b * 1024 * 16, w.DZ1);
  CNN_LAUNCHED();
  CNN_CHECK(wgrad(16, w.DZ1, w.A1, b * 1024, 16, 9, w.wpart, w.bpart, grad + kOffW1, grad + kOffB1, s));
#undef CNN_CHECK
#undef CNN_LAUNCHED
  return 0;
}

int cnn_adam_launch(float* params, const float* grad, float* m, float* v, int step, float lr, float beta1,
                    float beta2, float eps, void* stream) {
  const float c1 = 1.f - powf(beta1, static_cast<float>(step));
  const float c2 = 1.f - powf(beta2, static_cast<float>(step));
  adam_kernel<<<(kParams + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, grad, m, v, kParams, lr,
                                                                                   beta1, beta2, eps, c1, c2);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace cdct
