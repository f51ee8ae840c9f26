// Exact 8-point DCT-II through Chen's factorization (Eq. 3), in float32.
//
// T_C at the exact constants equals 2 C_8 (Sec. 3), so with C = C_8:
//   forward  B  = C A C^T  = (T A T^T) / 4
//   inverse  A' = C^T Bm C = (T^T Bm T) / 4
// One thread holds a whole 8x8 block; the row passes apply T (resp. T^T) to
// each row vector, the column passes to each column.  C is orthogonal, so
// the paper and transpose conventions coincide for this variant.
#include <cuda_runtime.h>

#include "block_kernels.cuh"

namespace cdct {
namespace {

typedef ParamsExact PE;

template <typename InT>
__device__ __forceinline__ void load_block_f(const BlockArgs& a, const BlockPos& s, float (&v)[8][8]) {
  const InT* img = static_cast<const InT*>(a.in) + static_cast<long long>(s.img) * a.in_bstride;
  int t[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    load_row<8, InT>(img, a, s.by * 8 + k, s.bx, t);
#pragma unroll
    for (int j = 0; j < 8; ++j) v[k][j] = static_cast<float>(t[j]);
  }
}

__device__ __forceinline__ void transpose8(float (&v)[8][8]) {
  float t[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) t[j][i] = v[i][j];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) v[i][j] = t[i][j];
}

// v holds rows on entry; on exit v[k][i] = 4 B(i, k) (column k of 4B)
__device__ __forceinline__ void forward8(float (&v)[8][8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) T8_apply<PE>(v[k]);     // rows: A T^T (x2)
  transpose8(v);
#pragma unroll
  for (int k = 0; k < 8; ++k) T8_apply<PE>(v[k]);     // columns: T (A T^T) (x2)
}

// v[k][i] = column k of (scaled) Bm on entry; rows of 16 A' on exit
__device__ __forceinline__ void inverse8(float (&v)[8][8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) T8t_apply<PE>(v[k]);    // columns: T^T Bm
  transpose8(v);
#pragma unroll
  for (int k = 0; k < 8; ++k) T8t_apply<PE>(v[k]);    // rows: (T^T Bm) T
}

__device__ __forceinline__ void mask8(const BlockArgs& a, float (&v)[8][8]) {
  const unsigned long long m = a.slab_mask[0];
#pragma unroll
  for (int k = 0; k < 8; ++k)
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (!((m >> (k * 8 + i)) & 1ull)) v[k][i] = 0.f;
}

template <typename InT>
__global__ void __launch_bounds__(kThreads) exact_fzi_kernel(const BlockArgs a) {
  const BlockPos s = block_pos<8>(a);
  float v[8][8];
  load_block_f<InT>(a, s, v);
  forward8(v);
  mask8(a, v);
  if (a.kept != nullptr && s.active) {
    float* dst = static_cast<float*>(a.kept) + (static_cast<long long>(s.img) * a.blocks_per_img + s.gb) * a.r;
    const unsigned long long m = a.slab_mask[0];
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if ((m >> (k * 8 + i)) & 1ull) dst[zigzag_pos(8, i, k)] = 0.25f * v[k][i];
  }
  inverse8(v);
  // v now holds 16 A' rows; a.scale = 1/16 turns it into pixels
  const double sse = store_rows_sse<8, InT>(a, s, v, a.partial != nullptr);
  if (a.partial != nullptr) cta_reduce_store(sse, a.partial);
}

template <typename InT>
__global__ void __launch_bounds__(kThreads) exact_forward_kernel(const BlockArgs a) {
  const BlockPos s = block_pos<8>(a);
  float v[8][8];
  load_block_f<InT>(a, s, v);
  forward8(v);
  if (!s.active) return;
  float* dst = static_cast<float*>(a.coeff) + (static_cast<long long>(s.img) * a.blocks_per_img + s.gb) * 64;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float4* d = reinterpret_cast<float4*>(dst + 8 * i);
    d[0] = make_float4(0.25f * v[0][i], 0.25f * v[1][i], 0.25f * v[2][i], 0.25f * v[3][i]);
    d[1] = make_float4(0.25f * v[4][i], 0.25f * v[5][i], 0.25f * v[6][i], 0.25f * v[7][i]);
  }
}

template <typename InT>
__global__ void __launch_bounds__(kThreads) exact_inverse_kernel(const BlockArgs a) {
  const BlockPos s = block_pos<8>(a);
  const float* src = static_cast<const float*>(a.coeff) + (static_cast<long long>(s.img) * a.blocks_per_img + s.gb) * 64;
  float v[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 q0 = __ldg(reinterpret_cast<const float4*>(src + 8 * i));
    const float4 q1 = __ldg(reinterpret_cast<const float4*>(src + 8 * i) + 1);
    v[0][i] = q0.x; v[1][i] = q0.y; v[2][i] = q0.z; v[3][i] = q0.w;
    v[4][i] = q1.x; v[5][i] = q1.y; v[6][i] = q1.z; v[7][i] = q1.w;
  }
  inverse8(v);
  store_rows_sse<8, InT>(a, s, v, false);
}

template <typename InT>
int launch_exact_fused(const BlockArgs& a, int batch, void* stream) {
  exact_fzi_kernel<InT><<<dim3(static_cast<unsigned>(batch) * a.ctas_per_img), kThreads, 0,
                          static_cast<cudaStream_t>(stream)>>>(a);
  return static_cast<int>(cudaGetLastError());
}
template <typename InT>
int launch_exact_forward(const BlockArgs& a, int batch, void* stream) {
  exact_forward_kernel<InT><<<dim3(static_cast<unsigned>(batch) * a.ctas_per_img), kThreads, 0,
                              static_cast<cudaStream_t>(stream)>>>(a);
  return static_cast<int>(cudaGetLastError());
}
template <typename InT>
int launch_exact_inverse(const BlockArgs& a, int batch, void* stream) {
  exact_inverse_kernel<InT><<<dim3(static_cast<unsigned>(batch) * a.ctas_per_img), kThreads, 0,
                              static_cast<cudaStream_t>(stream)>>>(a);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace

KernelSet kernels_exact8(int dtype) {
  KernelSet k;
  if (dtype == 0) {
    k.fused = launch_exact_fused<uint8_t>;
    k.forward = launch_exact_forward<uint8_t>;
    k.inverse = launch_exact_inverse<uint8_t>;
  } else {
    k.fused = launch_exact_fused<int16_t>;
    k.forward = launch_exact_forward<int16_t>;
    k.inverse = launch_exact_inverse<int16_t>;
  }
  return k;
}

}  // namespace cdct
