// Blockwise 2-D forward / zonal / inverse kernels (Sec. 5.1 pipeline).
//
// Work decomposition.  An image plane is cut into N x N blocks (padded by
// edge replication).  One thread owns a slab of W = 64 / N consecutive rows
// of one block (the whole block for N = 8), so P = N / W threads share a
// block and a 128-thread CTA owns 128 / P consecutive blocks of one image.
// Per block:
//   load W rows (128-bit loads) -> row pass -> [smem transpose] -> column
//   pass -> zonal mask -> inverse column pass -> [smem transpose] -> inverse
//   row pass -> float store (128-bit) + squared error.
// For N = 8 the block lives in one thread's registers and the "transposes"
// are register renames.  For N = 16 / 32 the transposes go through a
// per-block shared-memory tile whose 16-byte chunks are XOR-swizzled so that
// both the row-slab and the column-slab accesses are bank-conflict free.
//
// Arithmetic.  All integer stages are int32 adds (Jam<> in butterfly.cuh).
// The paper convention computes Y = T A U and Z = U Ym T; the transpose
// convention Y = T A T^T and Z = U Ym U^T.  The fused kernel carries U as
// W = 2U, so it holds 2Y (paper) or Y (transpose) and 4Z in both cases; the
// reconstruction is Z / N^2 = (4Z) * scale with scale = 1 / (4 N^2), a power
// of two, so the float result is the correctly rounded value of the exact
// rational reconstruction.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "butterfly.cuh"
#include "common.cuh"

namespace cdct {

template <int N>
struct Geo {
  static constexpr int W = 64 / N;              // rows (or columns) per thread
  static constexpr int P = N / W;               // threads per block
  static constexpr int BPC = kThreads / P;      // blocks per CTA
  static constexpr int CH = N / 4;              // 16-byte chunks per tile row
  // words per block tile; N = 16 tiles are offset by 16 words so that two
  // blocks served in one 8-thread phase of a 128-bit access hit disjoint banks
  static constexpr int STRIDE = N * N + (N == 16 ? 16 : 0);
  static constexpr int SMEM_WORDS = (P > 1) ? BPC * STRIDE : 4;
  static __device__ __forceinline__ int swz(int r) { return (r / W) & (CH - 1); }
};

// ---------------------------------------------------------------------------
// Global loads / stores
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 ldg_v4(const void* p) {
  return __ldg(reinterpret_cast<const uint4*>(p));
}
__device__ __forceinline__ uint2 ldg_v2(const void* p) {
  return __ldg(reinterpret_cast<const uint2*>(p));
}

__device__ __forceinline__ void unpack_i16(uint32_t u, int& lo, int& hi) {
  lo = static_cast<int>(u << 16) >> 16;
  hi = static_cast<int>(u) >> 16;
}

__device__ __forceinline__ int byte_of(uint32_t u, int k) {
  return static_cast<int>((u >> (8 * k)) & 0xffu);
}

// One row of N pixels starting at p (vector path, 16-byte aligned rows).
template <int N, typename InT>
__device__ __forceinline__ void load_row_vec(const InT* p, int (&x)[N]) {
  if constexpr (sizeof(InT) == 2) {
#pragma unroll
    for (int c = 0; c < N / 8; ++c) {
      const uint4 q = ldg_v4(p + 8 * c);
      unpack_i16(q.x, x[8 * c + 0], x[8 * c + 1]);
      unpack_i16(q.y, x[8 * c + 2], x[8 * c + 3]);
      unpack_i16(q.z, x[8 * c + 4], x[8 * c + 5]);
      unpack_i16(q.w, x[8 * c + 6], x[8 * c + 7]);
    }
  } else if constexpr (N == 8) {
    const uint2 q = ldg_v2(p);
#pragma unroll
    for (int k = 0; k < 4; ++k) { x[k] = byte_of(q.x, k); x[4 + k] = byte_of(q.y, k); }
  } else {
#pragma unroll
    for (int c = 0; c < N / 16; ++c) {
      const uint4 q = ldg_v4(p + 16 * c);
      const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int k = 0; k < 4; ++k) x[16 * c + 4 * t + k] = byte_of(w[t], k);
    }
  }
}

// One row, columns x0 .. x0+N-1 clamped to [0, width-1] (edge replication).
template <int N, typename InT>
__device__ __forceinline__ void load_row_clamped(const InT* row, int x0, int width, int (&x)[N]) {
#pragma unroll
  for (int j = 0; j < N; ++j) x[j] = static_cast<int>(__ldg(row + min(x0 + j, width - 1)));
}

template <int N, typename InT>
__device__ __forceinline__ void load_row(const InT* img, const BlockArgs& a, int gy, int bx,
                                         int (&x)[N]) {
  const InT* row = img + static_cast<long long>(min(gy, a.height - 1)) * a.in_pitch;
  const int x0 = bx * N;
  if (a.in_vec && x0 + N <= a.width) load_row_vec<N, InT>(row + x0, x);
  else load_row_clamped<N, InT>(row, x0, a.width, x);
}

// ---------------------------------------------------------------------------
// Slab transposes through shared memory (P > 1 only).
// rows -> cols: thread p holds rows p*W+k (k < W) of its block, all N
// columns; afterwards it holds columns p*W+k, all N rows (v[k][i]).
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ int* tile_of(int* smem, int lb) { return smem + lb * Geo<N>::STRIDE; }

template <int N>
__device__ __forceinline__ void rows_to_cols(int* smem, int lb, int p, int (&v)[Geo<N>::W][N]) {
  typedef Geo<N> G;
  if constexpr (G::P == 1) {
    int t[N][N];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int j = 0; j < N; ++j) t[j][i] = v[i][j];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int j = 0; j < N; ++j) v[i][j] = t[i][j];
  } else {
    int* tile = tile_of<N>(smem, lb);
#pragma unroll
    for (int k = 0; k < G::W; ++k) {
      const int r = p * G::W + k;
#pragma unroll
      for (int c = 0; c < G::CH; ++c) {
        const int cs = c ^ G::swz(r);
        *reinterpret_cast<int4*>(tile + r * N + 4 * cs) =
            make_int4(v[k][4 * c], v[k][4 * c + 1], v[k][4 * c + 2], v[k][4 * c + 3]);
      }
    }
    __syncwarp();
    // my columns p*W .. p*W+W-1 live in chunk (p*W)/4, at word offset (p*W)%4
    const int c = (p * G::W) >> 2, off = (p * G::W) & 3;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int* src = tile + i * N + 4 * (c ^ G::swz(i)) + off;
      if constexpr (G::W == 4) {
        const int4 q = *reinterpret_cast<const int4*>(src);
        v[0][i] = q.x; v[1][i] = q.y; v[2][i] = q.z; v[3][i] = q.w;
      } else {
        const int2 q = *reinterpret_cast<const int2*>(src);
        v[0][i] = q.x; v[1][i] = q.y;
      }
    }
    __syncwarp();
  }
}

template <int N>
__device__ __forceinline__ void cols_to_rows(int* smem, int lb, int p, int (&v)[Geo<N>::W][N]) {
  typedef Geo<N> G;
  if constexpr (G::P == 1) {
    rows_to_cols<N>(smem, lb, p, v);   // a square in-register transpose is its own inverse
  } else {
    int* tile = tile_of<N>(smem, lb);
    const int c = (p * G::W) >> 2, off = (p * G::W) & 3;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      int* dst = tile + i * N + 4 * (c ^ G::swz(i)) + off;
      if constexpr (G::W == 4) *reinterpret_cast<int4*>(dst) = make_int4(v[0][i], v[1][i], v[2][i], v[3][i]);
      else *reinterpret_cast<int2*>(dst) = make_int2(v[0][i], v[1][i]);
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < G::W; ++k) {
      const int r = p * G::W + k;
#pragma unroll
      for (int cc = 0; cc < G::CH; ++cc) {
        const int4 q = *reinterpret_cast<const int4*>(tile + r * N + 4 * (cc ^ G::swz(r)));
        v[k][4 * cc] = q.x; v[k][4 * cc + 1] = q.y; v[k][4 * cc + 2] = q.z; v[k][4 * cc + 3] = q.w;
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Per-convention 1-D operators.  CONV 0 = paper (Y = T A U, Z = U Ym T),
// CONV 1 = transpose (Y = T A T^T, Z = U Ym U^T).  A row pass applies the
// transpose of the right-hand matrix to each row vector.
// ---------------------------------------------------------------------------
template <int N, class P, int CONV>
struct Ops {
  static __device__ __forceinline__ void fwd_row(int (&x)[N]) {   // row * (2U) or row * T^T
    if constexpr (CONV == 0) Jam<N, P>::Wt(x); else Jam<N, P>::T(x);
  }
  static __device__ __forceinline__ void fwd_col(int (&x)[N]) { Jam<N, P>::T(x); }
  static __device__ __forceinline__ void inv_col(int (&x)[N]) { Jam<N, P>::W(x); }
  static __device__ __forceinline__ void inv_row(int (&x)[N]) {   // row * T or row * (2U)^T
    if constexpr (CONV == 0) Jam<N, P>::Tt(x); else Jam<N, P>::W(x);
  }
  // the fused forward result is (1 << FWD_SHIFT) * Y
  static constexpr int FWD_SHIFT = (CONV == 0) ? 1 : 0;
};

// ---------------------------------------------------------------------------
// Block bookkeeping
// ---------------------------------------------------------------------------
struct BlockPos {
  int img, lb, p, by, bx;
  long long gb;      // block index within the image
  bool active;
};

template <int N>
__device__ __forceinline__ BlockPos block_pos(const BlockArgs& a) {
  typedef Geo<N> G;
  BlockPos s;
  s.img = blockIdx.x / a.ctas_per_img;
  const int cta = blockIdx.x - s.img * a.ctas_per_img;
  s.lb = threadIdx.x / G::P;
  s.p = threadIdx.x - s.lb * G::P;
  long long gb = static_cast<long long>(cta) * G::BPC + s.lb;
  s.active = gb < a.blocks_per_img;
  if (!s.active) gb = a.blocks_per_img - 1;   // compute on a valid block, store nothing
  s.gb = gb;
  s.by = static_cast<int>(gb / a.nbx);
  s.bx = static_cast<int>(gb - static_cast<long long>(s.by) * a.nbx);
  return s;
}

template <int N>
__device__ __forceinline__ void apply_mask(const BlockArgs& a, int p, int (&v)[Geo<N>::W][N]) {
  const unsigned long long m = a.slab_mask[p];
#pragma unroll
  for (int k = 0; k < Geo<N>::W; ++k)
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (!((m >> (k * N + i)) & 1ull)) v[k][i] = 0;
}

// kept[blk][zz(i, j)] = Y(i, j) for the kept positions of this thread's columns
template <int N>
__device__ __forceinline__ void store_kept(const BlockArgs& a, const BlockPos& s,
                                           const int (&v)[Geo<N>::W][N], int shift) {
  const unsigned long long m = a.slab_mask[s.p];
  int32_t* dst = static_cast<int32_t*>(a.kept) +
                 (static_cast<long long>(s.img) * a.blocks_per_img + s.gb) * a.r;
#pragma unroll
  for (int k = 0; k < Geo<N>::W; ++k)
#pragma unroll
    for (int i = 0; i < N; ++i)
      if ((m >> (k * N + i)) & 1ull) dst[zigzag_pos(N, i, s.p * Geo<N>::W + k)] = v[k][i] >> shift;
}

// Store W rows of the reconstruction and accumulate the squared error
// against the (re-read) input pixels over the original H x W region.
template <int N, typename InT, typename VT>
__device__ __forceinline__ double store_rows_sse(const BlockArgs& a, const BlockPos& s,
                                                 const VT (&v)[Geo<N>::W][N], bool want_sse) {
  typedef Geo<N> G;
  const InT* img = static_cast<const InT*>(a.in) + static_cast<long long>(s.img) * a.in_bstride;
  float* out = a.out + static_cast<long long>(s.img) * a.out_bstride;
  const int x0 = s.bx * N;
  const bool full_x = x0 + N <= a.width;
  double total = 0.0;
#pragma unroll
  for (int k = 0; k < G::W; ++k) {
    const int gy = s.by * N + s.p * G::W + k;
    if (!s.active || gy >= a.height) continue;
    float rec[N];
#pragma unroll
    for (int j = 0; j < N; ++j) rec[j] = static_cast<float>(v[k][j]) * a.scale;
    float* orow = out + static_cast<long long>(gy) * a.out_pitch + x0;
    if (a.out_vec && full_x) {
#pragma unroll
      for (int c = 0; c < N / 4; ++c)
        __stcs(reinterpret_cast<float4*>(orow + 4 * c),
               make_float4(rec[4 * c], rec[4 * c + 1], rec[4 * c + 2], rec[4 * c + 3]));
    } else {
#pragma unroll
      for (int j = 0; j < N; ++j)
        if (x0 + j < a.width) orow[j] = rec[j];
    }
    if (want_sse) {
      int ref[N];
      load_row<N, InT>(img, a, gy, s.bx, ref);
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const float e = rec[j] - static_cast<float>(ref[j]);
        if (full_x || x0 + j < a.width) acc = fmaf(e, e, acc);
      }
      total += static_cast<double>(acc);
    }
  }
  return total;
}

// Deterministic CTA sum of one double per thread -> partial[blockIdx.x].
__device__ __forceinline__ void cta_reduce_store(double v, double* partial) {
  __shared__ double wsum[kThreads / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) t += wsum[w];
    partial[blockIdx.x] = t;
  }
}

// ---------------------------------------------------------------------------
// Kernels (integer variants)
// ---------------------------------------------------------------------------
template <int N, class P, int CONV, typename InT>
__global__ void __launch_bounds__(kThreads) fzi_kernel(const BlockArgs a) {
  typedef Geo<N> G;
  typedef Ops<N, P, CONV> O;
  __shared__ __align__(16) int smem[G::SMEM_WORDS];
  const BlockPos s = block_pos<N>(a);
  const InT* img = static_cast<const InT*>(a.in) + static_cast<long long>(s.img) * a.in_bstride;

  int v[G::W][N];
#pragma unroll
  for (int k = 0; k < G::W; ++k) load_row<N, InT>(img, a, s.by * N + s.p * G::W + k, s.bx, v[k]);
#pragma unroll
  for (int k = 0; k < G::W; ++k) O::fwd_row(v[k]);
  rows_to_cols<N>(smem, s.lb, s.p, v);
#pragma unroll
  for (int k = 0; k < G::W; ++k) O::fwd_col(v[k]);
  apply_mask<N>(a, s.p, v);
  if (a.kept != nullptr && s.active) store_kept<N>(a, s, v, O::FWD_SHIFT);
#pragma unroll
  for (int k = 0; k < G::W; ++k) O::inv_col(v[k]);
  cols_to_rows<N>(smem, s.lb, s.p, v);
#pragma unroll
  for (int k = 0; k < G::W; ++k) O::inv_row(v[k]);
  const double sse = store_rows_sse<N, InT>(a, s, v, a.partial != nullptr);
  if (a.partial != nullptr) cta_reduce_store(sse, a.partial);
}

template <int N, class P, int CONV, typename InT>
__global__ void __launch_bounds__(kThreads) forward_kernel(const BlockArgs a) {
  typedef Geo<N> G;
  typedef Ops<N, P, CONV> O;
  __shared__ __align__(16) int smem[G::SMEM_WORDS];
  const BlockPos s = block_pos<N>(a);
  const InT* img = static_cast<const InT*>(a.in) + static_cast<long long>(s.img) * a.in_bstride;
  int v[G::W][N];
#pragma unroll
  for (int k = 0; k < G::W; ++k) load_row<N, InT>(img, a, s.by * N + s.p * G::W + k, s.bx, v[k]);
#pragma unroll
  for (int k = 0; k < G::W; ++k) O::fwd_row(v[k]);
  rows_to_cols<N>(smem, s.lb, s.p, v);
#pragma unroll
  for (int k = 0; k < G::W; ++k) O::fwd_col(v[k]);
  if (!s.active) return;
  int32_t* dst = static_cast<int32_t*>(a.coeff) +
                 (static_cast<long long>(s.img) * a.blocks_per_img + s.gb) * (N * N) + s.p * G::W;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if constexpr (G::W == 8) {
      int4* d = reinterpret_cast<int4*>(dst + i * N);
      d[0] = make_int4(v[0][i] >> O::FWD_SHIFT, v[1][i] >> O::FWD_SHIFT, v[2][i] >> O::FWD_SHIFT, v[3][i] >> O::FWD_SHIFT);
      d[1] = make_int4(v[4][i] >> O::FWD_SHIFT, v[5][i] >> O::FWD_SHIFT, v[6][i] >> O::FWD_SHIFT, v[7][i] >> O::FWD_SHIFT);
    } else if constexpr (G::W == 4) {
      *reinterpret_cast<int4*>(dst + i * N) =
          make_int4(v[0][i] >> O::FWD_SHIFT, v[1][i] >> O::FWD_SHIFT, v[2][i] >> O::FWD_SHIFT, v[3][i] >> O::FWD_SHIFT);
    } else {
      *reinterpret_cast<int2*>(dst + i * N) = make_int2(v[0][i] >> O::FWD_SHIFT, v[1][i] >> O::FWD_SHIFT);
    }
  }
}

template <int N, class P, int CONV, typename InT>
__global__ void __launch_bounds__(kThreads) inverse_kernel(const BlockArgs a) {
  typedef Geo<N> G;
  typedef Ops<N, P, CONV> O;
  __shared__ __align__(16) int smem[G::SMEM_WORDS];
  const BlockPos s = block_pos<N>(a);
  const int32_t* src = static_cast<const int32_t*>(a.coeff) +
                       (static_cast<long long>(s.img) * a.blocks_per_img + s.gb) * (N * N) + s.p * G::W;
  int v[G::W][N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if constexpr (G::W == 8) {
      const int4 q0 = __ldg(reinterpret_cast<const int4*>(src + i * N));
      const int4 q1 = __ldg(reinterpret_cast<const int4*>(src + i * N) + 1);
      v[0][i] = q0.x; v[1][i] = q0.y; v[2][i] = q0.z; v[3][i] = q0.w;
      v[4][i] = q1.x; v[5][i] = q1.y; v[6][i] = q1.z; v[7][i] = q1.w;
    } else if constexpr (G::W == 4) {
      const int4 q = __ldg(reinterpret_cast<const int4*>(src + i * N));
      v[0][i] = q.x; v[1][i] = q.y; v[2][i] = q.z; v[3][i] = q.w;
    } else {
      const int2 q = __ldg(reinterpret_cast<const int2*>(src + i * N));
      v[0][i] = q.x; v[1][i] = q.y;
    }
  }
#pragma unroll
  for (int k = 0; k < G::W; ++k) O::inv_col(v[k]);
  cols_to_rows<N>(smem, s.lb, s.p, v);
#pragma unroll
  for (int k = 0; k < G::W; ++k) O::inv_row(v[k]);
  store_rows_sse<N, InT>(a, s, v, false);
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
template <int N, class P, int CONV, typename InT>
int launch_fused(const BlockArgs& a, int batch, void* stream) {
  const dim3 grid(static_cast<unsigned>(batch) * a.ctas_per_img);
  fzi_kernel<N, P, CONV, InT><<<grid, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(a);
  return static_cast<int>(cudaGetLastError());
}

template <int N, class P, int CONV, typename InT>
int launch_forward(const BlockArgs& a, int batch, void* stream) {
  const dim3 grid(static_cast<unsigned>(batch) * a.ctas_per_img);
  forward_kernel<N, P, CONV, InT><<<grid, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(a);
  return static_cast<int>(cudaGetLastError());
}

template <int N, class P, int CONV, typename InT>
int launch_inverse(const BlockArgs& a, int batch, void* stream) {
  const dim3 grid(static_cast<unsigned>(batch) * a.ctas_per_img);
  inverse_kernel<N, P, CONV, InT><<<grid, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(a);
  return static_cast<int>(cudaGetLastError());
}

template <int N, class P, int CONV>
KernelSet kernel_set_int(int dtype) {
  KernelSet k;
  if (dtype == 0) {
    k.fused = launch_fused<N, P, CONV, uint8_t>;
    k.forward = launch_forward<N, P, CONV, uint8_t>;
    k.inverse = launch_inverse<N, P, CONV, uint8_t>;
  } else {
    k.fused = launch_fused<N, P, CONV, int16_t>;
    k.forward = launch_forward<N, P, CONV, int16_t>;
    k.inverse = launch_inverse<N, P, CONV, int16_t>;
  }
  return k;
}

}  // namespace cdct
