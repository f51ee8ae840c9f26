// Persistent, bulk-copy pipelined fused kernel (forward -> zonal -> inverse
// -> squared error) for the integer variants.
//
// Work unit.  One segment of up to S = 128 / P consecutive blocks of one
// block row of one image: N pixel rows x (S * N) pixels, 8192 pixels when
// full.  The grid is persistent (a few CTAs per SM); CTA c takes units
// c, c + G, c + 2G, ... so every unit and its error partial are fixed.
//
// Pipeline.  The input rows of a unit are staged in shared memory by bulk
// asynchronous copies (cp.async.bulk, one per pixel row, issued by warp 0)
// into a STAGES-deep ring; an mbarrier per stage counts the landed bytes.
// While the CTA computes unit k, the copies for units k+1 .. k+STAGES-1 are
// in flight, so the HBM read stream never waits for the arithmetic.  Rows
// past the image bottom are fetched from the last row (edge replication);
// columns past the right edge are clamped when read from shared memory.
// The reconstruction goes straight from registers to HBM with 128-bit
// streaming stores; the squared error against the staged input is summed in
// float per thread and warp, and one double per unit is written.
//
// Zonal pruning.  With a compile-time r (RFIX > 0) only the JC x JC corner
// that contains the kept zig-zag positions is computed: the forward passes
// never produce the other outputs and the inverse passes see them as
// constant zeros, so the butterflies shrink to the adds that matter.  For
// N = 8 the whole mask is a compile-time constant.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "block_kernels.cuh"
#include "ptx.cuh"

namespace cdct {

// zig-zag cut: 1 + the highest row or column index among the first r
// positions (rows and columns can differ by one: an even partial diagonal
// starts at its bottom-left end, an odd one at its top-right end)
__host__ __device__ constexpr int zonal_extent(int n, int r) {
  int e = 0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (zigzag_pos(n, i, j) < r) {
        if (j + 1 > e) e = j + 1;
        if (i + 1 > e) e = i + 1;
      }
  return e;
}

__host__ __device__ constexpr unsigned long long slab_mask_ct(int n, int r, int p) {
  unsigned long long m = 0;
  const int w = 64 / n;
  for (int k = 0; k < w; ++k)
    for (int i = 0; i < n; ++i)
      if (zigzag_pos(n, i, p * w + k) < r) m |= 1ull << (k * n + i);
  return m;
}

template <int N, typename InT>
struct PipeGeo {
  typedef Geo<N> G;
  static constexpr int S = G::BPC;                       // blocks per unit
  static constexpr int WPX = S * N;                      // pixels per unit row
  static constexpr int ROWB = WPX * static_cast<int>(sizeof(InT));
  // staged row pitch; N = 32 rows are offset by 16 bytes so that the eight
  // rows read by one quarter warp fall in different bank groups
  static constexpr int ROWP = ROWB + (N == 32 ? 16 : 0);
  static constexpr int STAGE_BYTES = N * ROWP;
  static constexpr int TILE_STRIDE = (N == 16) ? N * N + 4 : N * N;  // words
  static constexpr int TILE_WORDS = (G::P > 1) ? S * TILE_STRIDE : 0;
  // lane -> (block in unit, slab) mapping
  static __device__ __forceinline__ void lane_map(int tid, int& lb, int& p) {
    if constexpr (N == 8) { lb = tid; p = 0; }
    else if constexpr (N == 16) {       // 8 blocks x 4 slabs per warp, slab-major
      const int w = tid >> 5, l = tid & 31;
      p = l >> 3; lb = w * 8 + (l & 7);
    } else {                            // 2 blocks x 16 slabs per warp, block-major
      lb = tid / 16; p = tid % 16;
    }
  }
  static constexpr size_t smem_bytes(int stages) {
    return static_cast<size_t>(stages) * STAGE_BYTES + static_cast<size_t>(TILE_WORDS) * 4;
  }
};

// Read row r (N pixels) of block lb from a staged unit with 128-bit shared
// loads.  `valid` = number of valid pixels of this block's rows (N unless
// the block crosses the right image edge, where columns are clamped to the
// last valid one).
template <int N, typename InT>
__device__ __forceinline__ void stage_read_row(const unsigned char* stage, int lb, int r, int valid, int (&x)[N]) {
  typedef PipeGeo<N, InT> PG;
  const InT* row = reinterpret_cast<const InT*>(stage + r * PG::ROWP) + lb * N;
  if (valid < N) {
#pragma unroll
    for (int j = 0; j < N; ++j) x[j] = static_cast<int>(row[min(j, valid - 1)]);
    return;
  }
  if constexpr (sizeof(InT) == 2) {
#pragma unroll
    for (int c = 0; c < N / 8; ++c) {      // 16-byte chunks of the block row
      const uint4 q = lds_v4(row + 8 * c);
      x[8 * c + 0] = sext_lo16(q.x); x[8 * c + 1] = sext_hi16(q.x);
      x[8 * c + 2] = sext_lo16(q.y); x[8 * c + 3] = sext_hi16(q.y);
      x[8 * c + 4] = sext_lo16(q.z); x[8 * c + 5] = sext_hi16(q.z);
      x[8 * c + 6] = sext_lo16(q.w); x[8 * c + 7] = sext_hi16(q.w);
    }
  } else if constexpr (N == 8) {
    const uint2 q = *reinterpret_cast<const uint2*>(row);
#pragma unroll
    for (int t = 0; t < 4; ++t) { x[t] = byte_u8(q.x, t); x[4 + t] = byte_u8(q.y, t); }
  } else {
#pragma unroll
    for (int c = 0; c < N / 16; ++c) {
      const uint4 q = lds_v4(row + 16 * c);
      const uint32_t wd[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int t = 0; t < 4; ++t) x[16 * c + 4 * e + t] = byte_u8(wd[e], t);
    }
  }
}

// The W rows of this thread's slab of block lb.
template <int N, typename InT>
__device__ __forceinline__ void stage_read_rows(const unsigned char* stage, int lb, int p, int valid,
                                                int (&v)[Geo<N>::W][N]) {
#pragma unroll
  for (int k = 0; k < Geo<N>::W; ++k) stage_read_row<N, InT>(stage, lb, p * Geo<N>::W + k, valid, v[k]);
}

// Slab transposes for the pipe kernels (tile per block at lb * TILE_STRIDE).
// JCW = number of leading columns (rows -> cols) or rows (cols -> rows) that
// carry data; the rest is known to be zero or unused.
template <int N, int JCW>
__device__ __forceinline__ void pipe_rows_to_cols(int* tiles, int lb, int p, int (&v)[Geo<N>::W][N]) {
  typedef Geo<N> G;
  if constexpr (G::P == 1) {
    rows_to_cols<N>(nullptr, 0, 0, v);
  } else {
    constexpr int TS = PipeGeo<N, int16_t>::TILE_STRIDE;
    constexpr int CHW = (JCW + 3) / 4;            // chunks that carry data
    int* tile = tiles + lb * TS;
#pragma unroll
    for (int k = 0; k < G::W; ++k) {
      const int r = p * G::W + k;
#pragma unroll
      for (int c = 0; c < CHW; ++c) {
        const int cs = c ^ G::swz(r);
        *reinterpret_cast<int4*>(tile + r * N + 4 * cs) =
            make_int4(v[k][4 * c], v[k][4 * c + 1], v[k][4 * c + 2], v[k][4 * c + 3]);
      }
    }
    __syncwarp();
    const int c = (p * G::W) >> 2, off = (p * G::W) & 3;
    const bool has = p * G::W < JCW;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int* src = tile + i * N + 4 * (c ^ G::swz(i)) + off;
      if constexpr (G::W == 4) {
        int4 q = has ? *reinterpret_cast<const int4*>(src) : make_int4(0, 0, 0, 0);
        v[0][i] = q.x; v[1][i] = q.y; v[2][i] = q.z; v[3][i] = q.w;
      } else {
        int2 q = has ? *reinterpret_cast<const int2*>(src) : make_int2(0, 0);
        v[0][i] = q.x; v[1][i] = q.y;
      }
    }
    __syncwarp();
  }
}

template <int N, int JCW>
__device__ __forceinline__ void pipe_cols_to_rows(int* tiles, int lb, int p, int (&v)[Geo<N>::W][N]) {
  typedef Geo<N> G;
  if constexpr (G::P == 1) {
    rows_to_cols<N>(nullptr, 0, 0, v);
  } else {
    constexpr int TS = PipeGeo<N, int16_t>::TILE_STRIDE;
    constexpr int CHW = (JCW + 3) / 4;
    int* tile = tiles + lb * TS;
    const int c = (p * G::W) >> 2, off = (p * G::W) & 3;
    if (p * G::W < JCW) {
#pragma unroll
      for (int i = 0; i < N; ++i) {
        int* dst = tile + i * N + 4 * (c ^ G::swz(i)) + off;
        if constexpr (G::W == 4) *reinterpret_cast<int4*>(dst) = make_int4(v[0][i], v[1][i], v[2][i], v[3][i]);
        else *reinterpret_cast<int2*>(dst) = make_int2(v[0][i], v[1][i]);
      }
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < G::W; ++k) {
      const int r = p * G::W + k;
#pragma unroll
      for (int cc = 0; cc < G::CH; ++cc) {
        if (cc < CHW) {
          const int4 q = *reinterpret_cast<const int4*>(tile + r * N + 4 * (cc ^ G::swz(r)));
          v[k][4 * cc] = q.x; v[k][4 * cc + 1] = q.y; v[k][4 * cc + 2] = q.z; v[k][4 * cc + 3] = q.w;
        } else {
          v[k][4 * cc] = 0; v[k][4 * cc + 1] = 0; v[k][4 * cc + 2] = 0; v[k][4 * cc + 3] = 0;
        }
      }
    }
    __syncwarp();
  }
}

// resident CTAs per SM the register allocation is sized for
template <int N>
struct PipeOcc { static constexpr int value = (N == 8) ? 4 : 3; };

template <int N, class P, int CONV, typename InT, int RFIX, int STAGES>
__global__ void __launch_bounds__(kThreads, PipeOcc<N>::value) fzi_pipe_kernel(const PipeArgs pa) {
  typedef Geo<N> G;
  typedef PipeGeo<N, InT> PG;
  typedef Ops<N, P, CONV> O;
  constexpr int W = G::W;
  // rows and columns that can hold kept coefficients
  constexpr int JC = RFIX > 0 ? zonal_extent(N, RFIX) : N;
  const BlockArgs& a = pa.b;

  extern __shared__ __align__(128) unsigned char smem[];
  int* tiles = reinterpret_cast<int*>(smem + STAGES * PG::STAGE_BYTES);
  __shared__ __align__(8) uint64_t full[STAGES];
  __shared__ float wsum[2][kThreads / 32];
  __shared__ int stop;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int lb, p;
  PG::lane_map(tid, lb, p);
  const uint64_t policy = policy_evict_first();
  const long long G_ = gridDim.x;
  const int es = static_cast<int>(sizeof(InT));

  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
    stop = 0;
  }
  __syncthreads();

  // warp 0 issues the copies of one unit into stage s
  auto issue = [&](long long u, int s) {
    const int img = static_cast<int>(u / pa.units_per_img);
    const long long rem = u - static_cast<long long>(img) * pa.units_per_img;
    const int by = static_cast<int>(rem / pa.units_per_row);
    const int seg = static_cast<int>(rem - static_cast<long long>(by) * pa.units_per_row);
    const int x0 = seg * PG::WPX;
    const uint32_t bytes = static_cast<uint32_t>(min(PG::WPX, a.width - x0) * es);
    if (lane == 0) mbar_arrive_expect_tx(&full[s], bytes * N);
    __syncwarp();
    if (lane < N) {
      const int gy = min(by * N + lane, a.height - 1);
      const InT* src = static_cast<const InT*>(a.in) + static_cast<long long>(img) * a.in_bstride +
                       static_cast<long long>(gy) * a.in_pitch + x0;
      bulk_g2s(smem + s * PG::STAGE_BYTES + lane * PG::ROWP, src, bytes, &full[s], policy);
    }
  };

  if (warp == 0) {
    for (int s = 0; s < STAGES; ++s) {
      const long long u = blockIdx.x + s * G_;
      if (u < pa.total_units) issue(u, s);
    }
  }

  for (int it = 0;; ++it) {
    const long long u = blockIdx.x + it * G_;
    if (u >= pa.total_units) break;
    const int s = it % STAGES;
    const uint32_t parity = static_cast<uint32_t>((it / STAGES) & 1);
    const bool ok = mbar_wait_bounded(&full[s], parity, pa.wait_limit);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(pa.err, 1);
        stop = 1;
      }
      break;
    }
    const unsigned char* stage = smem + s * PG::STAGE_BYTES;

    // unit -> image, block row, first block
    const int img = static_cast<int>(u / pa.units_per_img);
    const long long rem = u - static_cast<long long>(img) * pa.units_per_img;
    const int by = static_cast<int>(rem / pa.units_per_row);
    const int seg = static_cast<int>(rem - static_cast<long long>(by) * pa.units_per_row);
    const int bx = seg * PG::S + lb;
    const bool active = bx < a.nbx;
    const int x0 = bx * N;
    const int valid = active ? min(N, a.width - x0) : N;

    int v[W][N];
    stage_read_rows<N, InT>(stage, lb, p, valid, v);
    if (!active) {
#pragma unroll
      for (int k = 0; k < W; ++k)
#pragma unroll
        for (int j = 0; j < N; ++j) v[k][j] = 0;
    }

    // forward row pass; only columns < JC are ever used
#pragma unroll
    for (int k = 0; k < W; ++k) O::fwd_row(v[k]);
    pipe_rows_to_cols<N, JC>(tiles, lb, p, v);
#pragma unroll
    for (int k = 0; k < W; ++k) {
      O::fwd_col(v[k]);
#pragma unroll
      for (int i = JC; i < N; ++i) v[k][i] = 0;     // rows >= JC never kept
    }
    // zonal mask
    if constexpr (RFIX > 0 && G::P == 1) {
      constexpr unsigned long long m = slab_mask_ct(N, RFIX, 0);
#pragma unroll
      for (int k = 0; k < W; ++k)
#pragma unroll
        for (int i = 0; i < N; ++i)
          if (!((m >> (k * N + i)) & 1ull)) v[k][i] = 0;
    } else {
      const unsigned long long m = a.slab_mask[p];
#pragma unroll
      for (int k = 0; k < W; ++k)
#pragma unroll
        for (int i = 0; i < JC; ++i)
          if (!((m >> (k * N + i)) & 1ull)) v[k][i] = 0;
    }
    if (a.kept != nullptr && active) {
      BlockPos bp;
      bp.img = img; bp.lb = lb; bp.p = p; bp.by = by; bp.bx = bx;
      bp.gb = static_cast<long long>(by) * a.nbx + bx; bp.active = true;
      store_kept<N>(a, bp, v, O::FWD_SHIFT);
    }
#pragma unroll
    for (int k = 0; k < W; ++k) O::inv_col(v[k]);
    pipe_cols_to_rows<N, JC>(tiles, lb, p, v);
#pragma unroll
    for (int k = 0; k < W; ++k) O::inv_row(v[k]);

    // store the reconstruction, squared error against the staged input
    float acc = 0.f;
    float* out = a.out + static_cast<long long>(img) * a.out_bstride;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      const int gy = by * N + p * W + k;
      if (!active || gy >= a.height) continue;
      float rec[N];
#pragma unroll
      for (int j = 0; j < N; ++j) rec[j] = static_cast<float>(v[k][j]) * a.scale;
      float* orow = out + static_cast<long long>(gy) * a.out_pitch + x0;
      if (valid == N && a.out_vec) {
#pragma unroll
        for (int c = 0; c < N / 4; ++c)
          __stcs(reinterpret_cast<float4*>(orow + 4 * c),
                 make_float4(rec[4 * c], rec[4 * c + 1], rec[4 * c + 2], rec[4 * c + 3]));
      } else {
#pragma unroll
        for (int j = 0; j < N; ++j)
          if (j < valid) orow[j] = rec[j];
      }
      if (a.partial != nullptr) {
        int ref[1][N];
        stage_read_row<N, InT>(stage, lb, p * W + k, valid, ref[0]);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          if (j < valid) {
            const float e = rec[j] - static_cast<float>(ref[0][j]);
            acc = fmaf(e, e, acc);
          }
        }
      }
    }
    if (a.partial != nullptr) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
      if (lane == 0) wsum[it & 1][warp] = acc;
    }
    __syncthreads();   // the stage is consumed; wsum is complete
    if (tid == 0 && a.partial != nullptr) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < kThreads / 32; ++w) t += static_cast<double>(wsum[it & 1][w]);
      a.partial[u] = t;
    }
    if (warp == 0) {
      const long long un = u + STAGES * G_;
      if (un < pa.total_units) {
        fence_proxy_async_smem();
        issue(un, s);
      }
    }
  }

  __syncthreads();
  if (stop) {
    // a stage never completed: wait (bounded) for the copies that did get
    // issued so that none is still writing this CTA's shared memory
    if (tid == 0) {
      for (int s = 0; s < STAGES; ++s) {
        for (int ph = 0; ph < 2; ++ph) (void)mbar_wait_bounded(&full[s], ph, pa.wait_limit);
      }
    }
    __syncthreads();
  }
}

template <int N, class P, int CONV, typename InT, int RFIX, int STAGES>
int launch_pipe(const PipeArgs& pa, int grid, void* stream) {
  typedef PipeGeo<N, InT> PG;
  auto kern = fzi_pipe_kernel<N, P, CONV, InT, RFIX, STAGES>;
  const size_t smem = PG::smem_bytes(STAGES);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return static_cast<int>(e);
  kern<<<grid, kThreads, smem, static_cast<cudaStream_t>(stream)>>>(pa);
  return static_cast<int>(cudaGetLastError());
}

template <int N, class P, int CONV, typename InT, int RFIX, int STAGES>
int occupancy_pipe() {
  typedef PipeGeo<N, InT> PG;
  auto kern = fzi_pipe_kernel<N, P, CONV, InT, RFIX, STAGES>;
  const size_t smem = PG::smem_bytes(STAGES);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
    return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kThreads, smem) != cudaSuccess) return 0;
  return n;
}

}  // namespace cdct

namespace cdct {

// Launch the pipe kernel with the compile-time r among Rs that equals r, or
// the runtime-mask version; the grid is the resident CTA count, capped by
// the number of units.
template <int N, class P, int CONV, typename InT, int STAGES>
int pipe_launch_r(const PipeArgs& pa, int r, int num_sms, void* stream) {
  (void)r;
  static const int occ = occupancy_pipe<N, P, CONV, InT, 0, STAGES>();
  const long long cap = static_cast<long long>(num_sms) * (occ > 0 ? occ : 1);
  const int grid = static_cast<int>(pa.total_units < cap ? pa.total_units : cap);
  return launch_pipe<N, P, CONV, InT, 0, STAGES>(pa, grid, stream);
}

template <int N, class P, int CONV, typename InT, int STAGES, int R0, int... Rs>
int pipe_launch_r(const PipeArgs& pa, int r, int num_sms, void* stream) {
  if (r != R0) return pipe_launch_r<N, P, CONV, InT, STAGES, Rs...>(pa, r, num_sms, stream);
  static const int occ = occupancy_pipe<N, P, CONV, InT, R0, STAGES>();
  const long long cap = static_cast<long long>(num_sms) * (occ > 0 ? occ : 1);
  const int grid = static_cast<int>(pa.total_units < cap ? pa.total_units : cap);
  return launch_pipe<N, P, CONV, InT, R0, STAGES>(pa, grid, stream);
}

}  // namespace cdct
