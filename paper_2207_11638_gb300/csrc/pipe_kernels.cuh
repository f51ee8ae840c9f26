// Persistent, bulk-copy pipelined fused kernel (forward -> zonal -> inverse
// -> squared error) for the integer variants, N = 8, 16, 32.
//
// Work unit.  One segment of up to S consecutive blocks of one block row of
// one image, 8192 pixels when full (S = 128, 32, 8 for N = 8, 16, 32).  The
// grid is persistent; CTA c takes units c, c + G, c + 2G, ...  A uniform
// batch decodes a unit index with two fixed-point divisions.  A descriptor
// table (TABLE) gives each unit a 64-byte record, expanded on the host, which
// travels to shared memory with the stage's previous unit.
//
// Pipeline.  The input rows of a unit are staged in shared memory by bulk
// asynchronous copies (cp.async.bulk, one per pixel row, issued by one warp)
// into a STAGES-deep ring.  A "full" mbarrier per stage counts the landed
// bytes.  Every warp owns whole blocks, so a unit needs no CTA-wide barrier:
// a warp that finishes its part of a unit bumps the stage's counter in
// shared memory, and the last of the four refills the stage with the next
// unit.  No warp ever waits for another warp, only for its data.  All waits
// are bounded (clock64).
//
// Arithmetic.  The 2-D transform of an N x N block factors through the JAM
// recursion (Sec. 6, Eq. app_N) as
//     Y = P_N [T_8 G_ab R_8]_ab P_N^T,   G = F_N A F_N^T,
// where F_N is the cascade of M^add stages (the "fold": M^add_N, then
// M^add_{N/2} on each half), P_N the even/odd interleaves of M^per, G_ab the
// (N/8)^2 sub-blocks of size 8 x 8 of the folded block and R_8 the 8-point
// right factor (2U_8 or T_8^T).  The inverse is the mirror image: sub-block
// inverses, then the unfold F_N^T ( . ) F_N.  So N = 16 and 32 run the same
// register 8 x 8 core as N = 8, bracketed by fold / unfold adds that are
// exactly the M^add stages of the N-point butterflies:
//   N = 8:  one thread owns one block.
//   N = 16: a thread owns rows {p, 7-p, 8+p, 15-p} (p < 4) of a block; all
//           folds are thread-local; a warp-local exchange through shared
//           memory hands each of the 4 sub-blocks to one thread.
//   N = 32: a thread owns rows {p, 31-p} (p < 16); the horizontal folds and
//           the first vertical fold are thread-local; the second vertical
//           fold (and unfold) is done while reading the exchange buffer.
// The exchange buffers are XOR-swizzled so that every 128-bit access is
// bank-conflict free.
//
// Error.  The squared error against the staged input is summed per thread in
// float, reduced per warp, and one double per warp and unit is written.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "block_kernels.cuh"
#include "ptx.cuh"

namespace cdct {

template <int N, typename InT>
struct PipeGeo {
  static constexpr int P = N == 8 ? 1 : (N == 16 ? 4 : 16);   // threads per block
  static constexpr int S = kThreads / P;                       // blocks per unit
  static constexpr int WPX = S * N;                            // pixels per unit row
  static constexpr int ROWB = WPX * static_cast<int>(sizeof(InT));
  // staged row pitch; N = 32 rows are offset by 16 bytes so that the rows
  // p = 0..7 read by one quarter warp fall in different bank groups
  static constexpr int ROWP = ROWB + (N == 32 ? 16 : 0);
  static constexpr int STAGE_BYTES = N * ROWP;
  // exchange buffer (int32 words) per warp: N = 16: 8 blocks of 65 chunks;
  // N = 32: 2 blocks of 288 chunks (16-byte chunks, padded, see UnitBody)
  static constexpr int XCH_WARP_WORDS = (N == 8) ? 0 : (N == 16 ? 8 * 65 * 4 : 2 * 288 * 4);
  static constexpr int XCH_WORDS = XCH_WARP_WORDS * (kThreads / 32);
  static constexpr size_t smem_bytes(int stages) {
    return static_cast<size_t>(stages) * STAGE_BYTES + static_cast<size_t>(XCH_WORDS) * 4;
  }
};

// resident CTAs per SM the register allocation is sized for (N = 16 / 32
// with a one-stage ring fit four CTAs in shared memory, so they are built
// for four)
template <int N, int STAGES, int BODY = 0>
struct PipeOcc { static constexpr int value = (N == 8 || STAGES == 1 || BODY == 1) ? 4 : 3; };

// Read row r (N pixels) of the block whose row 0 starts at `sblk` in a staged
// unit (rows `spitch` bytes apart) with 128-bit shared loads.  `valid` = number of valid pixels of this block's rows (N unless
// the block crosses the right image edge, where columns are clamped to the
// last valid one).
template <int N, typename InT>
__device__ __forceinline__ void stage_read_row(const unsigned char* sblk, int spitch, int r, int valid,
                                               int (&x)[N]) {
  const InT* row = reinterpret_cast<const InT*>(sblk + r * spitch);
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

__device__ __forceinline__ void st_v4(int* p, const int* v) {
  *reinterpret_cast<int4*>(p) = make_int4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void ld_v4(const int* p, int* v) {
  const int4 q = *reinterpret_cast<const int4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}

// ---------------------------------------------------------------------------
// The 8 x 8 core: forward rows / columns, zonal mask, kept coefficients,
// inverse columns / rows.  v[i][j] holds row i on entry and on exit.  E is the
// compile-time extent (rows / columns >= E are never kept).  With a
// compile-time r (RFIX > 0) the bits that every sub-block keeps and the bits
// that no sub-block keeps are constants; only the rest are selected with the
// runtime mask m of this thread's sub-block q (for N = 8 none are left).  The
// constant zeros also prune the butterflies that consume them.
// ---------------------------------------------------------------------------
template <int N, class P, int CONV, int E, int RFIX>
__device__ __forceinline__ void core8(int (&v)[8][8], unsigned long long m, int32_t* kept, int q) {
  typedef Ops<8, P, CONV> O;
  constexpr unsigned long long ANY = RFIX > 0 ? sub_mask_any(N, RFIX) : ~0ull;
  constexpr unsigned long long ALL = RFIX > 0 ? sub_mask_all(N, RFIX) : 0ull;
#pragma unroll
  for (int i = 0; i < 8; ++i) O::fwd_row(v[i]);
  rows_to_cols<8>(nullptr, 0, 0, v);            // v[k][i]: column k
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k < E) {
      O::fwd_col(v[k]);
#pragma unroll
      for (int i = E; i < 8; ++i) v[k][i] = 0;
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) v[k][i] = 0;
    }
  }
#pragma unroll
  for (int k = 0; k < E; ++k)
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int bit = k * 8 + i;
      if (!((ANY >> bit) & 1ull)) v[k][i] = 0;
      else if (!((ALL >> bit) & 1ull) && !((m >> bit) & 1ull)) v[k][i] = 0;
    }
  if (kept != nullptr) {
#pragma unroll
    for (int k = 0; k < E; ++k)
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int bit = k * 8 + i;
        if (((ANY >> bit) & 1ull) && (((ALL >> bit) & 1ull) || ((m >> bit) & 1ull)))
          kept[zigzag_pos(N, sub_row_of(N, q, i), sub_col_of(N, q, k))] = v[k][i] >> O::FWD_SHIFT;
      }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (k < E) O::inv_col(v[k]);
  rows_to_cols<8>(nullptr, 0, 0, v);            // back to rows
#pragma unroll
  for (int i = 0; i < 8; ++i) O::inv_row(v[i]);
}

// ---------------------------------------------------------------------------
// Per-N unit bodies.  Each computes 4Z for the rows the thread owns, stores
// the reconstruction and returns the float squared error of those rows.
// ---------------------------------------------------------------------------
struct UnitPos {
  int img, by, bx;
  bool active;
  int valid;          // valid pixels of the block's rows
  bool fast;          // interior block: all N rows and columns valid, aligned output
  float* orow0;       // output row 0 of the block
  long long out_pitch;
  int height;
  const unsigned char* sblk;   // the block's staged row 0
  int spitch;                  // bytes between staged rows
  bool wrow;                   // the warp's blocks are adjacent in one block row
  const unsigned char* grow0;  // the block's input row 0 in global memory
  long long gpitch;            // bytes between input rows
};

// squared error of one staged row against a packed reconstruction row
template <int N, typename InT>
__device__ __forceinline__ f32x2 row_error(const InT* row, const f32x2 (&rec2)[N / 2], f32x2 acc2) {
  const f32x2 neg1 = pk2(-1.f, -1.f);
  if constexpr (sizeof(InT) == 2) {
    const f32x2 mg = pk2(-kMagicI16, -kMagicI16);
#pragma unroll
    for (int c = 0; c < N / 8; ++c) {
      const uint4 q = lds_v4(row + 8 * c);
      const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const f32x2 ref = add2(pk2(i16lo_magic(w[t]), i16hi_magic(w[t])), mg);
        const f32x2 e = fma2(ref, neg1, rec2[4 * c + t]);
        acc2 = fma2(e, e, acc2);
      }
    }
  } else {
    const f32x2 mg = pk2(-kMagicU8, -kMagicU8);
#pragma unroll
    for (int c = 0; c < N / 8; ++c) {
      const uint2 q = *reinterpret_cast<const uint2*>(row + 8 * c);
      const uint32_t w[2] = {q.x, q.y};
#pragma unroll
      for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const f32x2 ref = add2(pk2(u8_magic(w[t], 2 * h), u8_magic(w[t], 2 * h + 1)), mg);
          const f32x2 e = fma2(ref, neg1, rec2[4 * c + 2 * t + h]);
          acc2 = fma2(e, e, acc2);
        }
    }
  }
  return acc2;
}

// Store row r of the block's reconstruction (4Z in x) and return its squared
// error against the staged input.  Interior blocks take the check-free path.
template <int N, typename InT>
__device__ __forceinline__ float store_row(const BlockArgs& a, const UnitPos& up, int r, const int (&x)[N]) {
  const f32x2 sc2 = pk2(a.scale, a.scale);
  f32x2 rec2[N / 2];
#pragma unroll
  for (int j = 0; j < N / 2; ++j)
    rec2[j] = mul2(pk2(static_cast<float>(x[2 * j]), static_cast<float>(x[2 * j + 1])), sc2);
  float rec[N];
#pragma unroll
  for (int j = 0; j < N / 2; ++j) unpk2(rec2[j], rec[2 * j], rec[2 * j + 1]);
  const InT* row = reinterpret_cast<const InT*>(up.sblk + r * up.spitch);
  if (up.fast) {
    float* orow = up.orow0 + static_cast<long long>(r) * up.out_pitch;
    if (N == 8 && a.out_v8) {
      stcs_v8(orow, rec);                    // the whole block row: one full sector per thread
    } else {
#pragma unroll
      for (int c = 0; c < N / 4; ++c)
        __stcs(reinterpret_cast<float4*>(orow + 4 * c),
               make_float4(rec[4 * c], rec[4 * c + 1], rec[4 * c + 2], rec[4 * c + 3]));
    }
    if (a.partial == nullptr) return 0.f;
    float lo, hi;
    unpk2(row_error<N, InT>(row, rec2, pk2(0.f, 0.f)), lo, hi);
    return lo + hi;
  }
  const int gy = up.by * N + r;
  if (!up.active || gy >= up.height) return 0.f;
  float* orow = up.orow0 + static_cast<long long>(r) * up.out_pitch;
  if (up.valid == N && a.out_vec) {
#pragma unroll
    for (int c = 0; c < N / 4; ++c)
      __stcs(reinterpret_cast<float4*>(orow + 4 * c),
             make_float4(rec[4 * c], rec[4 * c + 1], rec[4 * c + 2], rec[4 * c + 3]));
  } else {
#pragma unroll
    for (int j = 0; j < N; ++j)
      if (j < up.valid) orow[j] = rec[j];
  }
  if (a.partial == nullptr) return 0.f;
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < N; ++j)
    if (j < up.valid) {
      const float e = rec[j] - static_cast<float>(row[min(j, up.valid - 1)]);
      acc = fmaf(e, e, acc);
    }
  return acc;
}

// Coalesced output of interior blocks (N = 16, 32).  Row r of the thread's
// block is converted as in store_row but written to the warp's staging
// buffer `obuf` (the exchange buffer, idle by then) instead of global
// memory; the warp then writes whole image-row segments of its adjacent
// blocks (copy_out).  For N = 32 copy_out also sums the squared error,
// reading the staged input of the pixels it writes.  Storing a block's rows straight from the threads
// that own them makes every 128-bit store touch one cache line per lane.
//   N = 16: staging row pitch 128 floats (8 blocks x 16), chunk c of block b
//           at physical chunk c ^ ((b >> 1) & 3) (conflict-free writes);
//   N = 32: staging row pitch 68 floats (2 blocks x 32 + 4 pad).
// N = 16 also returns the row's squared error against the staged input (its
// 32-byte rows read with 128-bit loads: fewer loads than copy_out's 64-bit
// ones); N = 32 leaves the error to copy_out and returns 0.
template <int N, typename InT>
__device__ __forceinline__ float stage_out_row(const BlockArgs& a, const UnitPos& up, int r, const int (&x)[N],
                                               float* obuf, int lbw) {
  const f32x2 sc2 = pk2(a.scale, a.scale);
  f32x2 rec2[N / 2];
#pragma unroll
  for (int j = 0; j < N / 2; ++j)
    rec2[j] = mul2(pk2(static_cast<float>(x[2 * j]), static_cast<float>(x[2 * j + 1])), sc2);
  float rec[N];
#pragma unroll
  for (int j = 0; j < N / 2; ++j) unpk2(rec2[j], rec[2 * j], rec[2 * j + 1]);
  float* orow = N == 16 ? obuf + r * 128 + lbw * 16 : obuf + r * 68 + lbw * 32;
  const int swz = N == 16 ? ((lbw >> 1) & 3) : 0;
#pragma unroll
  for (int c = 0; c < N / 4; ++c)
    *reinterpret_cast<float4*>(orow + 4 * (c ^ swz)) = make_float4(rec[4 * c], rec[4 * c + 1], rec[4 * c + 2],
                                                                   rec[4 * c + 3]);
  if (N != 16 || a.partial == nullptr) return 0.f;
  const InT* row = reinterpret_cast<const InT*>(up.sblk + r * up.spitch);
  float lo, hi;
  unpk2(row_error<N, InT>(row, rec2, pk2(0.f, 0.f)), lo, hi);
  return lo + hi;
}

// squared error of 4 staged pixels (columns col .. col + 3 of staged row `row`) against 4 reconstructions
template <typename InT>
__device__ __forceinline__ f32x2 quad_error(const InT* row, int col, float4 rec, f32x2 acc2) {
  const f32x2 neg1 = pk2(-1.f, -1.f);
  f32x2 r0, r1;
  if constexpr (sizeof(InT) == 2) {
    const uint2 q = *reinterpret_cast<const uint2*>(row + col);
    const f32x2 mg = pk2(-kMagicI16, -kMagicI16);
    r0 = add2(pk2(i16lo_magic(q.x), i16hi_magic(q.x)), mg);
    r1 = add2(pk2(i16lo_magic(q.y), i16hi_magic(q.y)), mg);
  } else {
    const uint32_t q = *reinterpret_cast<const uint32_t*>(row + col);
    const f32x2 mg = pk2(-kMagicU8, -kMagicU8);
    r0 = add2(pk2(u8_magic(q, 0), u8_magic(q, 1)), mg);
    r1 = add2(pk2(u8_magic(q, 2), u8_magic(q, 3)), mg);
  }
  const f32x2 e0 = fma2(r0, neg1, pk2(rec.x, rec.y));
  const f32x2 e1 = fma2(r1, neg1, pk2(rec.z, rec.w));
  acc2 = fma2(e0, e0, acc2);
  return fma2(e1, e1, acc2);
}

// Write the staged rows of the warp's blocks (N rows, each one contiguous
// segment of 8 x 16 or 2 x 32 floats starting at `base`, the first block's
// row 0) with 128-bit streaming stores that each cover whole cache lines,
// and return this lane's share of their squared error against the staged
// input (`sblk0`: the warp's first block's staged row 0) when `err`.
template <int N, typename InT>
__device__ __forceinline__ float copy_out(const float* obuf, float* base, long long pitch, int lane,
                                          const unsigned char* sblk0, int spitch, bool err) {
  f32x2 acc2 = pk2(0.f, 0.f);
  if constexpr (N == 16) {
    const int b = lane >> 2, c = (lane & 3) ^ ((b >> 1) & 3);
    const int col = b * 16 + c * 4;
#pragma unroll 4
    for (int r = 0; r < 16; ++r) {
      const float4 v = *reinterpret_cast<const float4*>(obuf + r * 128 + lane * 4);
      __stcs(reinterpret_cast<float4*>(base + r * pitch + b * 16 + c * 4), v);
      if (err) acc2 = quad_error<InT>(reinterpret_cast<const InT*>(sblk0 + r * spitch), col, v, acc2);
    }
  } else {
    const int h = lane >> 4, ch = lane & 15;
    const int col = ch * 4;
#pragma unroll 4
    for (int k = 0; k < 16; ++k) {
      const int r = 2 * k + h;
      const float4 v = *reinterpret_cast<const float4*>(obuf + r * 68 + ch * 4);
      __stcs(reinterpret_cast<float4*>(base + r * pitch + ch * 4), v);
      if (err) acc2 = quad_error<InT>(reinterpret_cast<const InT*>(sblk0 + r * spitch), col, v, acc2);
    }
  }
  float lo, hi;
  unpk2(acc2, lo, hi);
  return lo + hi;
}

__device__ __forceinline__ float* warp_base(float* orow0, int src_lane) {
  const unsigned long long v = reinterpret_cast<unsigned long long>(orow0);
  const unsigned lo = __shfl_sync(0xffffffffu, static_cast<unsigned>(v), src_lane);
  const unsigned hi = __shfl_sync(0xffffffffu, static_cast<unsigned>(v >> 32), src_lane);
  return reinterpret_cast<float*>((static_cast<unsigned long long>(hi) << 32) | lo);
}

__device__ __forceinline__ int32_t* kept_ptr(const BlockArgs& a, const UnitPos& up) {
  if (a.kept == nullptr || !up.active) return nullptr;
  return static_cast<int32_t*>(a.kept) +
         (static_cast<long long>(up.img) * a.blocks_per_img + static_cast<long long>(up.by) * a.nbx + up.bx) * a.r;
}

template <int N, class P, int CONV, typename InT, int RFIX>
struct UnitBody;

// N = 8: one thread, one block.
template <class P, int CONV, typename InT, int RFIX>
struct UnitBody<8, P, CONV, InT, RFIX> {
  static constexpr int E = RFIX > 0 ? zonal_extent(8, RFIX) : 8;
  static __device__ __forceinline__ int sub_block(int /*lane*/) { return 0; }
  static __device__ __forceinline__ float run(const BlockArgs& a, const UnitPos& up, const unsigned char* stage,
                                              int* /*xch*/, int /*lane*/, int lb, unsigned long long mask) {
    int v[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i) stage_read_row<8, InT>(up.sblk, up.spitch, i, up.valid, v[i]);
    core8<8, P, CONV, E, RFIX>(v, mask, kept_ptr(a, up), 0);
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc += store_row<8, InT>(a, up, i, v[i]);
    return acc;
  }
};

// N = 16: thread (block lb, p < 4) owns rows {p, 7-p, 8+p, 15-p}; in the
// core it owns sub-block s = p.  Exchange buffer per block: 16-byte chunks
// [s 4][row 8][ch 2], blocks 65 chunks apart (the odd stride spreads the 8
// blocks of one quarter warp over all bank groups).
template <class P, int CONV, typename InT, int RFIX>
struct UnitBody<16, P, CONV, InT, RFIX> {
  static constexpr int E = RFIX > 0 ? (zonal_extent(16, RFIX) + 1) / 2 : 8;
  // word offset of chunk (s, row, ch) within a block
  static constexpr int off(int s, int row, int ch) { return 4 * ((s * 8 + row) * 2 + ch); }
  static __device__ __forceinline__ int sub_block(int lane) { return lane >> 3; }
  static __device__ __forceinline__ float run(const BlockArgs& a, const UnitPos& up, const unsigned char* stage,
                                              int* xch, int lane, int lb, unsigned long long mask) {
    const int p = lane >> 3, lbw = lane & 7;
    int* buf = xch + lbw * 65 * 4;
    int* rp = buf + 8 * p;              // row p of every sub-block
    int* rq = buf + 8 * (7 - p);        // row 7-p
    {
      const int rows[4] = {p, 7 - p, 8 + p, 15 - p};
      int h[4][2][8];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        int x[16];
        stage_read_row<16, InT>(up.sblk, up.spitch, rows[t], up.valid, x);
        madd<16>(x, h[t][0], h[t][1]);                 // horizontal fold
      }
      // vertical fold: top row p = r0 + r3, top row 7-p = r1 + r2,
      //                bottom row p = r1 - r2, bottom row 7-p = r0 - r3
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        int g[4][8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          g[0][j] = h[0][b][j] + h[3][b][j];
          g[1][j] = h[1][b][j] + h[2][b][j];
          g[2][j] = h[1][b][j] - h[2][b][j];
          g[3][j] = h[0][b][j] - h[3][b][j];
        }
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          st_v4(rp + off(0 + b, 0, ch), &g[0][4 * ch]);
          st_v4(rq + off(0 + b, 0, ch), &g[1][4 * ch]);
          st_v4(rp + off(2 + b, 0, ch), &g[2][4 * ch]);
          st_v4(rq + off(2 + b, 0, ch), &g[3][4 * ch]);
        }
      }
    }
    __syncwarp();
    {
      const int s = p;
      int* sb = buf + off(s, 0, 0);
      int v[8][8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) ld_v4(sb + off(0, i, ch), &v[i][4 * ch]);
      __syncwarp();
      core8<16, P, CONV, E, RFIX>(v, mask, kept_ptr(a, up), s);
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) st_v4(sb + off(0, i, ch), &v[i][4 * ch]);
    }
    __syncwarp();
    int xr[4][16];                          // rows p, 15-p, 7-p, 8+p
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      // vertical unfold: half 0 yields rows p and 15-p, half 1 rows 7-p and 8+p:
      //   x_p = top_p + bot_{7-p},      x_{15-p} = top_p - bot_{7-p}
      //   x_{7-p} = top_{7-p} + bot_p,  x_{8+p} = top_{7-p} - bot_p
      int* rt = half == 0 ? rp : rq;
      int* rb = half == 0 ? rq : rp;
      int lo_s[8], hi_s[8], lo_d[8], hi_d[8];
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        int t[8], u[8];
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          ld_v4(rt + off(0 + b, 0, ch), &t[4 * ch]);
          ld_v4(rb + off(2 + b, 0, ch), &u[4 * ch]);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (b == 0) { lo_s[j] = t[j] + u[j]; lo_d[j] = t[j] - u[j]; }
          else { hi_s[j] = t[j] + u[j]; hi_d[j] = t[j] - u[j]; }
        }
      }
      madd_join<16>(lo_s, hi_s, xr[2 * half]);        // horizontal unfold
      madd_join<16>(lo_d, hi_d, xr[2 * half + 1]);
    }
    __syncwarp();                           // every unfold read of the exchange buffer is done
    float acc = 0.f;
    if (up.wrow && __all_sync(0xffffffffu, up.fast)) {
      float* obuf = reinterpret_cast<float*>(xch);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int r0 = (k >> 1) == 0 ? p : 7 - p;
        acc += stage_out_row<16, InT>(a, up, (k & 1) ? 15 - r0 : r0, xr[k], obuf, lbw);
      }
      __syncwarp();
      copy_out<16, InT>(obuf, warp_base(up.orow0, 0), up.out_pitch, lane, nullptr, 0, false);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int r0 = (k >> 1) == 0 ? p : 7 - p;
        acc += store_row<16, InT>(a, up, (k & 1) ? 15 - r0 : r0, xr[k]);
      }
    }
    __syncwarp();
    return acc;
  }
};

// N = 32: thread (block lb, p < 16) owns rows {p, 31-p}; in the core it owns
// sub-block q = hr*8 + ar*4 + c (hr: first vertical fold half, ar: second,
// c = h*2 + a' for the two horizontal folds).  Per block, 288 chunks of 16
// bytes hold, in turn:
//   layout 1 (after the first vertical fold): chunk (hr*16 + row)*9 + 2c + ch
//   layout 2 (core output):                    chunk q*17 + 2row + (row >> 2) + ch
// The odd strides / the pad chunk after row 3 make every access pattern
// below bank-conflict free with plain base + constant addressing.
template <class P, int CONV, typename InT, int RFIX>
struct UnitBody<32, P, CONV, InT, RFIX> {
  static constexpr int E = RFIX > 0 ? (zonal_extent(32, RFIX) + 3) / 4 : 8;
  static constexpr int l2(int q, int row, int ch) { return 4 * (q * 17 + 2 * row + (row >> 2) + ch); }
  static __device__ __forceinline__ int sub_block(int lane) { return lane & 15; }
  static __device__ __forceinline__ float run(const BlockArgs& a, const UnitPos& up, const unsigned char* stage,
                                              int* xch, int lane, int lb, unsigned long long mask) {
    const int p = lane & 15, lbw = lane >> 4;
    int* buf = xch + lbw * 288 * 4;
    {
      int hc[2][4][8];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        int x[32], lo[16], hi[16];
        stage_read_row<32, InT>(up.sblk, up.spitch, t == 0 ? p : 31 - p, up.valid, x);
        madd<32>(x, lo, hi);                       // horizontal fold, first level
        madd<16>(lo, hc[t][0], hc[t][1]);          // second level: c = h*2 + a'
        madd<16>(hi, hc[t][2], hc[t][3]);
      }
      // first vertical fold: half 0 row p = x_p + x_{31-p}, half 1 row 15-p = x_p - x_{31-p}
      int* w0 = buf + 4 * (p * 9);
      int* w1 = buf + 4 * ((16 + 15 - p) * 9);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        int s0[8], s1[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) { s0[j] = hc[0][c][j] + hc[1][c][j]; s1[j] = hc[0][c][j] - hc[1][c][j]; }
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          st_v4(w0 + 4 * (2 * c + ch), &s0[4 * ch]);
          st_v4(w1 + 4 * (2 * c + ch), &s1[4 * ch]);
        }
      }
    }
    __syncwarp();
    {
      const int q = p, hr = q >> 3, ar = (q >> 2) & 1, c = q & 3;
      const int sgn = ar ? -1 : 1;
      // second vertical fold within half hr:
      //   ar = 0: row i = H[i] + H[15-i];  ar = 1: row i = H[7-i] - H[8+i]
      const int* hb = buf + 4 * (hr * 16 * 9 + 2 * c);
      const int* pa = hb + 4 * 9 * (ar ? 7 : 0);
      const int* pb = hb + 4 * 9 * (ar ? 8 : 15);
      const int step = ar ? -4 * 9 : 4 * 9;        // pa walks down (ar = 1) or up, pb the other way
      int v[8][8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          int t[4], u[4];
          ld_v4(pa + 4 * ch, t);
          ld_v4(pb + 4 * ch, u);
#pragma unroll
          for (int e = 0; e < 4; ++e) v[i][4 * ch + e] = t[e] + sgn * u[e];
        }
        pa += step;
        pb -= step;
      }
      __syncwarp();
      core8<32, P, CONV, E, RFIX>(v, mask, kept_ptr(a, up), q);
      int* qb = buf + l2(q, 0, 0);
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) st_v4(qb + l2(0, i, ch), &v[i][4 * ch]);
    }
    __syncwarp();
    // second vertical unfold (within each half), then the first:
    //   H[m] = top_m + bot_{7-m} (m < 8),  H[8+k] = top_{7-k} - bot_k
    //   x_p = H0[p] + H1[15-p],  x_{31-p} = H0[p] - H1[15-p]
    int hc0[4][8], hc1[4][8];
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int m = hr == 0 ? p : 15 - p;
      const int rt = m < 8 ? m : 15 - m, rb = m < 8 ? 7 - m : m - 8;
      const int sg = m < 8 ? 1 : -1;
      const int* bt = buf + l2(0, rt, 0);
      const int* bb = buf + l2(0, rb, 0);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int qt = hr * 8 + c, qb = hr * 8 + 4 + c;
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          int t[4], u[4];
          ld_v4(bt + 4 * (qt * 17 + ch), t);
          ld_v4(bb + 4 * (qb * 17 + ch), u);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (hr == 0) hc0[c][4 * ch + e] = t[e] + sg * u[e];
            else hc1[c][4 * ch + e] = t[e] + sg * u[e];
          }
        }
      }
    }
    __syncwarp();                                  // every unfold read of the exchange buffer is done
    float acc = 0.f;
    const bool co = up.wrow && __all_sync(0xffffffffu, up.fast);
    float* obuf = reinterpret_cast<float*>(xch);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      int cc[4][8];
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int j = 0; j < 8; ++j) cc[c][j] = t == 0 ? hc0[c][j] + hc1[c][j] : hc0[c][j] - hc1[c][j];
      int lo[16], hi[16], x[32];
      madd_join<16>(cc[0], cc[1], lo);             // horizontal unfold, second level
      madd_join<16>(cc[2], cc[3], hi);
      madd_join<32>(lo, hi, x);                    // first level
      if (co) stage_out_row<32, InT>(a, up, t == 0 ? p : 31 - p, x, obuf, lbw);
      else acc += store_row<32, InT>(a, up, t == 0 ? p : 31 - p, x);
    }
    if (co) {
      __syncwarp();
      acc = copy_out<32, InT>(obuf, warp_base(up.orow0, 0), up.out_pitch, lane, up.sblk - lbw * 32 * sizeof(InT),
                              up.spitch, a.partial != nullptr);
    }
    __syncwarp();
    return acc;
  }
};

}  // namespace cdct

#include "sep_body.cuh"

namespace cdct {

// The fold + 8 x 8 core bodies behind the interface the kernel uses:
// exchange words per warp, a constant area in shared memory (none), a
// per-thread context (the zonal mask of the thread's sub-block) and run().
template <int N, class P, int CONV, typename InT, int RFIX>
struct FoldBody {
  typedef UnitBody<N, P, CONV, InT, RFIX> B;
  static constexpr int XCH_WARP_WORDS = PipeGeo<N, InT>::XCH_WARP_WORDS;
  static constexpr int CONST_WORDS = 0;
  struct Ctx {
    unsigned long long mask;
  };
  static __device__ __forceinline__ void init_const(float*, int) {}
  static __device__ __forceinline__ void init(Ctx& c, const BlockArgs& a, int lane, const float*) {
    c.mask = a.slab_mask[B::sub_block(lane)];
  }
  static constexpr bool EARLY_RELEASE = false;
  // block of the unit a thread works on: N = 8 one per thread; N = 16 eight
  // per warp (lane & 7); N = 32 two per warp (lane >> 4)
  static __device__ __forceinline__ int lane_block(int warp, int lane) {
    return N == 8 ? warp * 32 + lane : (N == 16 ? warp * 8 + (lane & 7) : warp * 2 + (lane >> 4));
  }
  template <class Rel>
  static __device__ __forceinline__ float run(const BlockArgs& a, const UnitPos& up, int* xch, const float*, int lane,
                                              const Ctx& cx, Rel&& release) {
    const float acc = B::run(a, up, nullptr, xch, lane, 0, cx.mask);
    release();                                  // the stage is read to the end (squared error)
    return acc;
  }
};

// BODY 0: fold + 8 x 8 core (any r, both conventions, kept coefficients);
// BODY 1: separable packed passes (N = 16, 32; paper convention; r = RFIX).
template <int N, class P, int CONV, typename InT, int RFIX, int BODY>
struct BodySel {
  typedef FoldBody<N, P, CONV, InT, RFIX> type;
};
template <class P, typename InT, int RFIX>
struct BodySel<32, P, 0, InT, RFIX, 1> {
  typedef SepBody32<P, InT, RFIX> type;
};
template <class P, typename InT, int RFIX>
struct BodySel<16, P, 0, InT, RFIX, 1> {
  typedef SepBody16<P, InT, RFIX> type;
};

template <int N, typename InT, class Body>
constexpr size_t pipe_smem_bytes(int stages) {
  return static_cast<size_t>(stages) * PipeGeo<N, InT>::STAGE_BYTES +
         static_cast<size_t>(Body::XCH_WARP_WORDS * (kThreads / 32) + Body::CONST_WORDS) * 4;
}

// ---------------------------------------------------------------------------
// Unit decoding: image, block row and segment of unit u, with the image's
// geometry, for a uniform batch (BlockArgs) or a descriptor table.
// ---------------------------------------------------------------------------
template <typename InT>
struct UnitSrc {
  int img, by, seg;
  int pack, rows;         // block rows per unit (1 unless packed) and those this unit covers
  const InT* in;          // first pixel of the image
  long long in_pitch;
  int width, height, nbx;
  float* out;             // first reconstructed pixel of the image
  long long out_pitch;
};

template <int N, typename InT>
__device__ __forceinline__ void decode_record(const UnitDesc& m, UnitSrc<InT>& d) {
  d.img = m.img;
  d.in = static_cast<const InT*>(m.data);
  d.in_pitch = m.pitch;
  d.width = m.width;
  d.height = m.height;
  d.nbx = (d.width + N - 1) / N;
  d.out = m.recon;
  d.out_pitch = m.recon_pitch;
  d.pack = pack_rows(d.nbx, PipeGeo<N, InT>::S);
  d.by = m.by;
  d.seg = m.seg;
  d.rows = m.rows;
}

template <int N, typename InT, bool TABLE>
__device__ __forceinline__ void decode_unit(const PipeArgs& pa, uint32_t u, UnitSrc<InT>& d) {
  typedef PipeGeo<N, InT> PG;
  const BlockArgs& a = pa.b;
  if constexpr (!TABLE) {
    uint32_t rem, seg;
    d.img = static_cast<int>(fdiv(u, pa.div_img, rem));
    d.by = static_cast<int>(fdiv(rem, pa.div_row, seg));
    d.seg = static_cast<int>(seg);
    d.in = static_cast<const InT*>(a.in) + static_cast<long long>(d.img) * a.in_bstride;
    d.in_pitch = a.in_pitch;
    d.width = a.width;
    d.height = a.height;
    d.nbx = a.nbx;
    d.out = a.out + static_cast<long long>(d.img) * a.out_bstride;
    d.out_pitch = a.out_pitch;
    d.pack = 1;
    d.rows = 1;
  } else {
    // the unit's record, expanded on the host
    decode_record<N, InT>(pa.unit_map[u], d);
  }
}

// ---------------------------------------------------------------------------
// The persistent kernel
// ---------------------------------------------------------------------------
template <int N, class P, int CONV, typename InT, int RFIX, int STAGES, bool TABLE, int BODY>
__global__ void __launch_bounds__(kThreads, PipeOcc<N, STAGES, BODY>::value) fzi_pipe_kernel(const PipeArgs pa) {
  typedef PipeGeo<N, InT> PG;
  typedef typename BodySel<N, P, CONV, InT, RFIX, BODY>::type Body;
  constexpr int NW = kThreads / 32;
  const BlockArgs& a = pa.b;

  extern __shared__ __align__(128) unsigned char smem[];
  int* xch_all = reinterpret_cast<int*>(smem + STAGES * PG::STAGE_BYTES);
  float* cbuf = reinterpret_cast<float*>(xch_all + Body::XCH_WARP_WORDS * NW);
  __shared__ __align__(8) uint64_t full[STAGES];
  __shared__ int done[STAGES];           // warps that finished the stage's current unit
  // Descriptor tables.  usrc[s]: the decoded unit of stage s, written by the
  // warp that issues its copies before its arrival on full[s] (so it is
  // visible once the stage is).  rec[s]: the record of the unit that stage s
  // takes next, bulk-copied with the current unit's pixels (and counted by
  // full[s]), so that the refill decodes from shared memory.  Uniform
  // batches decode with two fixed-point divisions instead.
  __shared__ UnitSrc<InT> usrc[TABLE ? STAGES : 1];
  __shared__ __align__(16) UnitDesc rec[TABLE ? STAGES : 1];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int* xch = xch_all + warp * Body::XCH_WARP_WORDS;
  // block of this thread within the unit
  const int lb = Body::lane_block(warp, lane);
  // input lines are read once (evict first), or a second time from L2 by a
  // body that releases its stage early and reads the pixels it compares with
  // from global memory (normal priority)
  const uint64_t policy = Body::EARLY_RELEASE ? policy_evict_normal() : policy_evict_first();
  const long long G_ = gridDim.x;
  const int es = static_cast<int>(sizeof(InT));

  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      done[s] = 0;
    }
    fence_mbar_init();
  }
  Body::init_const(cbuf, tid);
  __syncthreads();

  // one whole warp issues the copies of unit u, decoded into d, into stage s
  auto issue = [&](long long u, int s, const UnitSrc<InT>& d) {
    const int x0 = d.seg * PG::WPX;
    const uint32_t bytes = static_cast<uint32_t>(min(PG::WPX, d.width - x0) * es);
    // the record of the unit this stage takes after u
    const long long un = u + STAGES * G_;
    const uint32_t rec_bytes = (TABLE && un < pa.total_units) ? static_cast<uint32_t>(sizeof(UnitDesc)) : 0u;
    if (pa.drop_copies) {          // failure-detection test: the stage's phase can never complete
      if (lane == 0) mbar_arrive_expect_tx(&full[s], 16u);
      __syncwarp();
      return;
    }
    if (d.pack == 1) {
      if (lane == 0) {
        if constexpr (TABLE) usrc[s] = d;
        mbar_arrive_expect_tx(&full[s], bytes * N + rec_bytes);
      }
      __syncwarp();
      if (TABLE && lane == 31 && rec_bytes != 0) bulk_g2s(&rec[s], pa.unit_map + un, rec_bytes, &full[s], policy);
      if (lane < N) {
        const int gy = min(d.by * N + lane, d.height - 1);
        const InT* src = d.in + static_cast<long long>(gy) * d.in_pitch + x0;
        bulk_g2s(smem + s * PG::STAGE_BYTES + lane * PG::ROWP, src, bytes, &full[s], policy);
      }
    } else {
      // packed narrow image: rows * N whole pixel rows, `bytes` apart (a multiple of 16);
      // rows * N * bytes <= N * ROWB <= STAGE_BYTES since pack * nbx <= S
      const int nr = d.rows * N;
      if (lane == 0) {
        if constexpr (TABLE) usrc[s] = d;
        mbar_arrive_expect_tx(&full[s], bytes * nr + rec_bytes);
      }
      __syncwarp();
      if (TABLE && lane == 31 && rec_bytes != 0) bulk_g2s(&rec[s], pa.unit_map + un, rec_bytes, &full[s], policy);
      for (int j = lane; j < nr; j += 32) {
        const int gy = min(d.by * N + j, d.height - 1);
        const InT* src = d.in + static_cast<long long>(gy) * d.in_pitch;
        bulk_g2s(smem + s * PG::STAGE_BYTES + j * bytes, src, bytes, &full[s], policy);
      }
    }
  };

  if (warp == 0) {
    for (int s = 0; s < STAGES; ++s) {
      const long long u = blockIdx.x + s * G_;
      if (u < pa.total_units) {
        UnitSrc<InT> d;
        decode_unit<N, InT, TABLE>(pa, static_cast<uint32_t>(u), d);
        issue(u, s, d);
      }
    }
  }

  // the thread's part of a unit (and so its zonal mask or factors) is the same in every unit
  typename Body::Ctx ctx;
  Body::init(ctx, a, lane, cbuf);

  bool failed = false;
  int it = 0;
  for (;; ++it) {
    const long long u = blockIdx.x + it * G_;
    if (u >= pa.total_units) break;
    const int s = it % STAGES;
    const uint32_t parity = static_cast<uint32_t>((it / STAGES) & 1);
    const bool landed = mbar_wait_bounded(&full[s], parity, pa.wait_limit);
    if (!__all_sync(0xffffffffu, landed)) { failed = true; break; }   // the warp stops as one
    const unsigned char* stage = smem + s * PG::STAGE_BYTES;

    UnitSrc<InT> d;
    if constexpr (TABLE) d = usrc[s];
    else decode_unit<N, InT, false>(pa, static_cast<uint32_t>(u), d);
    UnitPos up;
    up.img = d.img;
    up.out_pitch = d.out_pitch;
    up.height = d.height;
    if (d.pack == 1) {
      up.by = d.by;
      up.bx = d.seg * PG::S + lb;
      up.active = up.bx < d.nbx;
      up.sblk = stage + lb * N * es;
      up.spitch = PG::ROWP;
      up.wrow = true;
    } else {
      // packed: block lb is block (lb % nbx) of block row by + lb / nbx
      const int k = lb / d.nbx;
      up.by = d.by + k;
      up.bx = lb - k * d.nbx;
      up.active = k < d.rows;
      up.spitch = d.width * es;
      up.sblk = up.active ? stage + k * N * up.spitch + up.bx * N * es : stage;
      const int wb = N == 16 ? 8 : (N == 32 ? 2 : 1);       // blocks per warp
      const int lb0 = warp * wb;                              // the warp's first block
      up.wrow = (lb0 % d.nbx) + wb <= d.nbx;
    }
    up.valid = up.active ? min(N, d.width - up.bx * N) : N;
    up.fast = up.active && up.valid == N && a.out_vec && (up.by + 1) * N <= d.height;
    up.orow0 = d.out + static_cast<long long>(up.by) * N * d.out_pitch + up.bx * N;
    up.gpitch = d.in_pitch * es;
    up.grow0 = reinterpret_cast<const unsigned char*>(d.in + static_cast<long long>(up.by) * N * d.in_pitch + up.bx * N);

    // release the stage (the body calls this once it has read the stage for
    // the last time); the last warp to do so refills it with unit u + STAGES*G
    auto release = [&]() {
      __syncwarp();
      int last = 0;
      if (lane == 0) {
        __threadfence_block();                 // this warp's reads of the stage come first
        last = atomicAdd(&done[s], 1) == NW - 1;
        if (last) {
          done[s] = 0;
          __threadfence_block();
        }
      }
      last = __shfl_sync(0xffffffffu, last, 0);
      if (last) {
        const long long un = u + STAGES * G_;
        if (un < pa.total_units) {
          UnitSrc<InT> dn;
          if constexpr (TABLE) decode_record<N, InT>(rec[s], dn);   // landed with unit u
          else decode_unit<N, InT, false>(pa, static_cast<uint32_t>(un), dn);
          fence_proxy_async_smem();    // the warps' reads of the stage (and of rec[s]) before the copies
          issue(un, s, dn);
        }
      }
    };
    float acc = Body::run(a, up, xch, cbuf, lane, ctx, release);

    if (a.partial != nullptr) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
      if (lane == 0) a.partial[u * NW + warp] = static_cast<double>(acc);
    }
  }

  if (failed) {
    if (lane == 0) atomicOr(pa.err, 1);
    // the units this warp leaves unfinished get NaN partials, so that a PSNR
    // reduced from them shows the failure instead of stale values
    if (a.partial != nullptr && lane == 0)
      for (long long uk = blockIdx.x + static_cast<long long>(it) * G_; uk < pa.total_units; uk += G_)
        a.partial[uk * NW + warp] = __longlong_as_double(0x7FF8000000000000ll);
    // wait (bounded) for copies that may still be landing in this CTA's
    // stages, so that none writes shared memory after the CTA exits
    for (int k = 0; k < STAGES; ++k) {
      const int itk = it + k;
      const long long uk = blockIdx.x + static_cast<long long>(itk) * G_;
      if (uk >= pa.total_units) break;
      (void)mbar_wait_bounded(&full[itk % STAGES], static_cast<uint32_t>((itk / STAGES) & 1), pa.wait_limit);
    }
  }
}

template <int N, class P, int CONV, typename InT, int RFIX, int STAGES, bool TABLE, int BODY = 0>
int launch_pipe(const PipeArgs& pa, int num_sms, int ctas_per_sm, void* stream) {
  typedef typename BodySel<N, P, CONV, InT, RFIX, BODY>::type Body;
  auto kern = fzi_pipe_kernel<N, P, CONV, InT, RFIX, STAGES, TABLE, BODY>;
  const size_t smem = pipe_smem_bytes<N, InT, Body>(STAGES);
  static int occ = -1;   // resident CTAs per SM (same for every GPU this library targets)
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return static_cast<int>(e);
  if (occ < 0) {
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kThreads, smem);
    if (e != cudaSuccess) return static_cast<int>(e);
    occ = n > 0 ? n : 1;
  }
  const int per_sm = (ctas_per_sm > 0 && ctas_per_sm < occ) ? ctas_per_sm : occ;
  const long long cap = static_cast<long long>(num_sms) * per_sm;
  const int grid = static_cast<int>(pa.total_units < cap ? pa.total_units : cap);
  if (grid <= 0) return 0;
  kern<<<grid, kThreads, smem, static_cast<cudaStream_t>(stream)>>>(pa);
  return static_cast<int>(cudaGetLastError());
}

// Launch with the compile-time r among Rs that equals r, or the runtime-mask
// version.
template <int N, class P, int CONV, typename InT, int STAGES, bool TABLE>
int pipe_launch_r(const PipeArgs& pa, int r, int num_sms, int ctas_per_sm, void* stream) {
  (void)r;
  return launch_pipe<N, P, CONV, InT, 0, STAGES, TABLE>(pa, num_sms, ctas_per_sm, stream);
}

template <int N, class P, int CONV, typename InT, int STAGES, bool TABLE, int R0, int... Rs>
int pipe_launch_r(const PipeArgs& pa, int r, int num_sms, int ctas_per_sm, void* stream) {
  if (r != R0) return pipe_launch_r<N, P, CONV, InT, STAGES, TABLE, Rs...>(pa, r, num_sms, ctas_per_sm, stream);
  return launch_pipe<N, P, CONV, InT, R0, STAGES, TABLE>(pa, num_sms, ctas_per_sm, stream);
}

// The separable packed body where it applies (paper convention, r = RFIX,
// no kept-coefficient output), else the fold + core body at its own depth.
template <int N, class P, typename InT, int RFIX, int STAGES, bool TABLE>
bool pipe_try_sep(const PipeArgs& pa, int conv, int r, int num_sms, int ctas_per_sm, void* stream, int& rc) {
  if (conv != 0 || r != RFIX || pa.b.kept != nullptr) return false;
  rc = launch_pipe<N, P, 0, InT, RFIX, STAGES, TABLE, 1>(pa, num_sms, ctas_per_sm, stream);
  return true;
}

}  // namespace cdct
