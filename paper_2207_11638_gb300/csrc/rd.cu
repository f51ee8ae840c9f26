// Exhaustive rate-distortion quadtree search over 32 x 32 regions.
//
// For every region and every quantiser step q the kernel evaluates the 21
// blocks of the three transform sizes (one 32 x 32, four 16 x 16, sixteen
// 8 x 8) and picks the cheapest of the 17 quadtrees (32 | each quadrant 16 or
// four 8s).  Per block, in exact integer arithmetic:
//   Y  = T A U                         forward transform, paper convention (Sec. 5.1)
//   L  = round(B / q),  B = diag(s) Y diag(s)^-1 / N   with the paper's round() (Sec. 3),
//        decided exactly: |L| = max{k : 4 Y^2 d_j >= (2k - 1)^2 N^2 q^2 d_i}, d = diag(T T^T)
//   Y' = N q L c,  c_ij = round(2^F sqrt(d_i / d_j))   fixed-point dequantisation, F = 12
//   Z' = U Y' T                        reconstruction times 2^F N^2
//   D  = sum (2^F N^2 A - Z')^2        pixel-domain squared error (valid pixels only)
//   R  = 1 + (last zig-zag position + 1) + sum over nonzero L of (2 floor(log2 |L|) + 2)
//   J' = (32 / N)^4 D + lambda' R,     lambda' = kappa q^2 2^(2F + 20)
// all held as unsigned 128-bit integers, so the labels are exact.
//
// Layout: one warp per region.  The region is staged in shared memory as
// int32 (row pitch 33 words); transposes go through a 32 x 33 int64 buffer.
// A lane owns one column, then one row, of the region: the column and row
// passes apply the N-point butterflies to the 32 / N segments of its line.
// Forward passes run in int32 (|2Y| < 2^27 for |A| <= 1023), the decoder in
// int64 (|Z'| < 2^56).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "butterfly.cuh"
#include "common.cuh"

namespace cdct {
namespace {

typedef unsigned __int128 u128;

constexpr int kRdWarps = 4;                  // regions (warps) per CTA
constexpr int kRdThreads = 32 * kRdWarps;
constexpr int kRdFrac = 12;                  // F
constexpr int kPitch = 33;                   // padded row pitch (words)

struct RdSmem {
  int d[3][32];                              // d_i for N = 32, 16, 8
  // dequantisation scales c_ij, rows padded to N + 1 words: lane i reads row i, so an
  // unpadded row pitch of N would put all lanes of a read in one bank
  int c32[32 * 33], c16[16 * 17], c8[8 * 9];
  float sd[3][32];                           // sqrt(d_j) (first guesses of the quantiser only)
  int a[kRdWarps][32 * kPitch];              // regions
  long long buf[kRdWarps][32 * kPitch];      // transposes
  u128 cost[kRdWarps][4][21];                // block costs per q: [0] 32, [1..4] 16, [5..20] 8
};

__device__ __forceinline__ int size_slot(int n) { return n == 32 ? 0 : (n == 16 ? 1 : 2); }
__device__ __forceinline__ int cost_base(int n) { return n == 32 ? 0 : (n == 16 ? 1 : 5); }

__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int m) {
  unsigned long long lo = static_cast<unsigned long long>(v), hi = static_cast<unsigned long long>(v >> 64);
  lo = __shfl_xor_sync(0xffffffffu, lo, m);
  hi = __shfl_xor_sync(0xffffffffu, hi, m);
  return (static_cast<u128>(hi) << 64) | lo;
}

// The level's magnitude from the float estimate alone, where that is safe.
// With x = |y| sqrt(d_j) / (n q sqrt(d_i)) the level is floor(x + 1/2).  t =
// fmaf(float(|y|), est, 1/2) carries seven correctly rounded operations
// (sqrtf twice, two products, the reciprocal, the conversion of |y| and the
// fma), so |t - (x + 1/2)| <= 7.01 * 2^-24 (x + 1/2) < 2^-21 t (1 + 2^-20).  If
// t - d and t + d, d = t 2^-20, round down to one integer, floor(t) is the
// level; otherwise `exact` is set and the integer test must decide.
__device__ __forceinline__ int quant_guess(unsigned a, float est, bool& exact) {
  const float t = fmaf(static_cast<float>(a), est, 0.5f);
  const float d = t * 0x1p-20f;
  const float lo = floorf(t - d);
  exact = lo != floorf(t + d);
  return static_cast<int>(lo);
}

// The level's magnitude by the integer test, from a guess within one of it
__device__ __forceinline__ int quant_settle(unsigned a, unsigned dj, unsigned long long unit, int k) {
  const unsigned long long lhs = (static_cast<unsigned long long>(a) * a) * (4ull * dj);
  if (k < 0) k = 0;
  while (static_cast<unsigned long long>(2 * k + 1) * static_cast<unsigned>(2 * k + 1) * unit <= lhs) ++k;
  while (k > 0 && static_cast<unsigned long long>(2 * k - 1) * static_cast<unsigned>(2 * k - 1) * unit > lhs) --k;
  return k;
}

// Key of zig-zag position (i, j) of an n x n block that orders like the
// position itself: 64 (i + j) + (i on odd diagonals, 63 - i on even ones), as
// zig-zag runs down odd diagonals and up even ones.  key_pos inverts it.
__device__ __forceinline__ int zz_key_even_j(int i) { return 64 * i + ((i & 1) ? i : 63 - i); }
__device__ __forceinline__ int zz_key_odd_j(int i) { return 64 * i + ((i & 1) ? 63 - i : i); }
__device__ __forceinline__ int key_pos(int n, int key) {
  if (key < 0) return -1;
  const int d = key >> 6, sub = key & 63;
  const int i = (d & 1) ? sub : 63 - sub;
  return zigzag_pos(n, i, d - i);
}

__device__ __forceinline__ int level_bits(int l) {
  const unsigned a = static_cast<unsigned>(l < 0 ? -l : l);
  return a == 0 ? 0 : 2 * (31 - __clz(a)) + 2;
}

struct RdKernelArgs {
  const void* in;
  long long pitch, bstride;
  int width, height, tiles_x, tiles_per_img;
  long long n_regions;
  int nq;
  int q[4];
  unsigned long long lam_lo[4], lam_hi[4];
  unsigned char* labels;                     // [nq][n_regions]
  unsigned long long* part_cost;             // [nq][n_regions][17][2] or null
  int tables[3 * 32 + 32 * 32 + 16 * 16 + 8 * 8];   // d[3][32], c32, c16, c8 (by value)
  // subset search (mode 1): region numbers and their count (device)
  const long long* subset;
  const long long* subset_count;
  long long max_count;
  // evaluation of given labels (mode 2)
  const unsigned char* in_labels;            // [nq][n_regions]
  unsigned long long* ev_cost;               // [nq][n_regions][2]: J' of the labelled partition
  unsigned long long* ev_dist;               // [nq][n_regions][2]: its distortion on the J' scale, or null
  int* ev_bits;                              // [nq][n_regions]: its rate in bits, or null
};

// Per-block distortion and rate, kept beside the costs when labels are evaluated.
struct RdEvalSmem {
  u128 dist[kRdWarps][4][21];
  int bits[kRdWarps][4][21];
};

// One transform size for the region staged in sa; block costs into cost[qi][...].
// `need`: bit qi set when step qi needs this size (all steps when searching);
// `edist` / `ebits` (evaluation only, else null) receive each block's scaled
// distortion and rate.
template <int N, class P>
__device__ __forceinline__ void rd_size(const RdKernelArgs& ka, const RdSmem& sm, const int* sa, long long* buf,
                                        u128 (*cost)[21], int lane, int vrows, int vcols, unsigned need,
                                        u128 (*edist)[21], int (*ebits)[21]) {
  constexpr int S = 32 / N;
  int* b32 = reinterpret_cast<int*>(buf);
  const int* dd = sm.d[N == 32 ? 0 : (N == 16 ? 1 : 2)];
  const int* cc = N == 32 ? sm.c32 : (N == 16 ? sm.c16 : sm.c8);
  // forward, columns: T applied to each N-segment of column `lane`
  {
    int col[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) col[r] = sa[r * kPitch + lane];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      int x[N];
#pragma unroll
      for (int k = 0; k < N; ++k) x[k] = col[s * N + k];
      Jam<N, P>::T(x);
#pragma unroll
      for (int k = 0; k < N; ++k) col[s * N + k] = x[k];
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) b32[r * kPitch + lane] = col[r];
  }
  __syncwarp();
  // forward, rows: (T A) U = ((2U)^T applied to each row) / 2
  int y[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) y[c] = b32[lane * kPitch + c];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    int x[N];
#pragma unroll
    for (int k = 0; k < N; ++k) x[k] = y[s * N + k];
    Jam<N, P>::Wt(x);
#pragma unroll
    for (int k = 0; k < N; ++k) y[s * N + k] = x[k] >> 1;     // 2Y is even: exact
  }
  __syncwarp();
  const int i = lane % N;                   // block-local row of this lane's coefficients
  const int di = dd[i];
  const float* sdj = sm.sd[N == 32 ? 0 : (N == 16 ? 1 : 2)];
  for (int qi = 0; qi < ka.nq; ++qi) {
    if (!((need >> qi) & 1u)) continue;      // warp-uniform
    const int q = ka.q[qi];
    const unsigned long long unit = static_cast<unsigned long long>(N * N) * static_cast<unsigned>(q * q) *
                                    static_cast<unsigned>(di);
    const float est_i = 1.0f / (static_cast<float>(N * q) * sdj[i]);
    int rate[S], last[S];
#pragma unroll
    for (int s = 0; s < S; ++s) { rate[s] = 0; last[s] = -1; }
    const int key_e = zz_key_even_j(i), key_o = zz_key_odd_j(i);
    // quantise, count bits, dequantise (row `lane`); last[] holds zig-zag keys here
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      const int j = c % N;
      const unsigned a = static_cast<unsigned>(y[c] < 0 ? -y[c] : y[c]);
      bool exact;
      int k = quant_guess(a, sdj[j] * est_i, exact);
      if (__any_sync(0xffffffffu, exact)) {       // warp-uniform: rare
        if (exact) k = quant_settle(a, static_cast<unsigned>(dd[j]), unit, k);
      }
      const int l = y[c] < 0 ? -k : k;
      rate[c / N] += level_bits(k);
      if (k != 0) last[c / N] = max(last[c / N], ((j & 1) ? key_o : key_e) + 64 * j);
      // |N q L| < 2^23 and c < 2^16: one 32 x 32 -> 64-bit product
      long long yq = 0;
      if (k != 0) yq = static_cast<long long>(N * q * l) * cc[i * (N + 1) + j];
      buf[lane * kPitch + c] = yq;
    }
    __syncwarp();
    // inverse, columns: (2U) Y'
    {
      long long col[32];
#pragma unroll
      for (int r = 0; r < 32; ++r) col[r] = buf[r * kPitch + lane];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        long long x[N];
#pragma unroll
        for (int k = 0; k < N; ++k) x[k] = col[s * N + k];
        Jam<N, P>::W(x);
#pragma unroll
        for (int k = 0; k < N; ++k) col[s * N + k] = x[k];
      }
#pragma unroll
      for (int r = 0; r < 32; ++r) buf[r * kPitch + lane] = col[r];
    }
    __syncwarp();
    // inverse, rows: ((2U) Y') T = 2 Z'; squared error against 2^F N^2 A
    // squared errors below 2^58 are summed in 64 bits (at most 32 of them per
    // segment: below 2^63), larger ones in 128 bits
    u128 dist[S];
    unsigned long long dsmall[S];
#pragma unroll
    for (int s = 0; s < S; ++s) dist[s] = 0, dsmall[s] = 0;
    {
      long long row[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) row[c] = buf[lane * kPitch + c];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        long long x[N];
#pragma unroll
        for (int k = 0; k < N; ++k) x[k] = row[s * N + k];
        Jam<N, P>::Tt(x);
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const int c = s * N + k;
          const long long ref = static_cast<long long>(sa[lane * kPitch + c]) * (N * N) << kRdFrac;
          const long long e = ref - (x[k] >> 1);              // 2Z' is even: exact
          const unsigned long long ae = static_cast<unsigned long long>(e < 0 ? -e : e);
          if (lane < vrows && c < vcols) {
            if (ae >> 29) dist[s] += static_cast<u128>(ae) * ae;
            else dsmall[s] += static_cast<unsigned long long>(static_cast<unsigned>(ae)) * static_cast<unsigned>(ae);
          }
        }
      }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) dist[s] += dsmall[s];
    __syncwarp();
    // per block: sum over its N lanes (aligned groups), then the cost
#pragma unroll
    for (int s = 0; s < S; ++s) {
#pragma unroll
      for (int m = N / 2; m >= 1; m >>= 1) {
        if (m >= 32) continue;
        dist[s] += shfl_xor_u128(dist[s], m);
        rate[s] += __shfl_xor_sync(0xffffffffu, rate[s], m);
        last[s] = max(last[s], __shfl_xor_sync(0xffffffffu, last[s], m));
      }
    }
    if (i == 0) {
      const u128 lam = (static_cast<u128>(ka.lam_hi[qi]) << 64) | ka.lam_lo[qi];
      constexpr unsigned long long kScale = (32 / N) * (32 / N) * (32 / N) * (32 / N);
      const int br = lane / N;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const int bits = 1 + (key_pos(N, last[s]) + 1) + rate[s];
        cost[qi][cost_base(N) + br * S + s] = dist[s] * kScale + lam * static_cast<unsigned>(bits);
        if (edist != nullptr) {
          edist[qi][cost_base(N) + br * S + s] = dist[s] * kScale;
          ebits[qi][cost_base(N) + br * S + s] = bits;
        }
      }
    }
    __syncwarp();
  }
}

// MODE 0: search every region; 1: search the listed regions; 2: evaluate the
// given labels, one transform size EVN per launch (32 first: it initialises
// each output with the partition's split flags; 16 and 8 then add their
// blocks).  One size per launch keeps every warp of an SM in the same code:
// with the three sizes mixed across warps, instruction fetch dominated.
template <class P, typename InT, int MODE, int EVN = 0>
__global__ void __launch_bounds__(kRdThreads, 3) rd_kernel(const RdKernelArgs ka) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RdSmem& sm = *reinterpret_cast<RdSmem*>(smem_raw);
  RdEvalSmem* ev = MODE == 2 ? reinterpret_cast<RdEvalSmem*>(smem_raw + sizeof(RdSmem)) : nullptr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // constant tables into shared memory (per-lane indexed reads)
  {
    for (int t = threadIdx.x; t < 3 * 32; t += kRdThreads) {
      sm.d[t / 32][t % 32] = ka.tables[t];
      sm.sd[t / 32][t % 32] = sqrtf(static_cast<float>(ka.tables[t]));
    }
    const int* c = ka.tables + 3 * 32;
    for (int t = threadIdx.x; t < 32 * 32; t += kRdThreads) sm.c32[(t >> 5) * 33 + (t & 31)] = c[t];
    for (int t = threadIdx.x; t < 16 * 16; t += kRdThreads) sm.c16[(t >> 4) * 17 + (t & 15)] = c[1024 + t];
    for (int t = threadIdx.x; t < 8 * 8; t += kRdThreads) sm.c8[(t >> 3) * 9 + (t & 7)] = c[1024 + 256 + t];
  }
  __syncthreads();
  int* sa = sm.a[warp];
  long long* buf = sm.buf[warp];
  u128 (*cost)[21] = sm.cost[warp];
  u128 (*edist)[21] = MODE == 2 ? ev->dist[warp] : nullptr;
  int (*ebits)[21] = MODE == 2 ? ev->bits[warp] : nullptr;
  const unsigned all = (1u << ka.nq) - 1u;
  long long count = ka.n_regions;
  if (MODE == 1) {
    count = *ka.subset_count;
    count = count < ka.max_count ? count : ka.max_count;
  }
  const long long stride = static_cast<long long>(gridDim.x) * kRdWarps;
  for (long long k = static_cast<long long>(blockIdx.x) * kRdWarps + warp; k < count; k += stride) {
    const long long reg = MODE == 1 ? ka.subset[k] : k;
    if (reg < 0 || reg >= ka.n_regions) continue;
    const int img = static_cast<int>(reg / ka.tiles_per_img);
    const int t = static_cast<int>(reg - static_cast<long long>(img) * ka.tiles_per_img);
    const int ty = t / ka.tiles_x, tx = t - (t / ka.tiles_x) * ka.tiles_x;
    const int y0 = ty * 32, x0 = tx * 32;
    const int vrows = min(32, ka.height - y0), vcols = min(32, ka.width - x0);
    // sizes each step needs: all of them when searching, the labelled partition's when evaluating
    unsigned need32 = all, need16 = all, need8 = all;
    int lab_q = 0;
    if (MODE == 2) {
      need32 = need16 = need8 = 0;
      for (int qi = 0; qi < ka.nq; ++qi) {
        int l = ka.in_labels[static_cast<long long>(qi) * ka.n_regions + reg];
        l = l < 17 ? l : 0;
        if (lane == qi) lab_q = l;
        if (l == 0) need32 |= 1u << qi;
        else {
          if (l - 1 != 15) need16 |= 1u << qi;
          if (l - 1 != 0) need8 |= 1u << qi;
        }
      }
      // a region that uses this size for any step is coded at every step: all warps then
      // run the same code as the search (a per-step skip made warps diverge and fetch-bound)
      need32 = (EVN == 32 && need32) ? all : 0;
      need16 = (EVN == 16 && need16) ? all : 0;
      need8 = (EVN == 8 && need8) ? all : 0;
      if (EVN != 32 && (need16 | need8) == 0) continue;   // nothing of this size to add (warp-uniform)
    }
    if ((need32 | need16 | need8) != 0) {
      // stage the region (edge replicated beyond the image), lane = column
      const InT* src = static_cast<const InT*>(ka.in) + img * ka.bstride;
      const int gx = x0 + min(lane, vcols - 1);
#pragma unroll 4
      for (int r = 0; r < 32; ++r) {
        const int gy = y0 + min(r, vrows - 1);
        sa[r * kPitch + lane] = static_cast<int>(src[gy * ka.pitch + gx]);
      }
      __syncwarp();
    }
    if ((MODE != 2 || EVN == 32) && need32)
      rd_size<32, P>(ka, sm, sa, buf, cost, lane, vrows, vcols, need32, edist, ebits);
    if ((MODE != 2 || EVN == 16) && need16)
      rd_size<16, P>(ka, sm, sa, buf, cost, lane, vrows, vcols, need16, edist, ebits);
    if ((MODE != 2 || EVN == 8) && need8)
      rd_size<8, P>(ka, sm, sa, buf, cost, lane, vrows, vcols, need8, edist, ebits);
    if (MODE == 2) {
      // this size's share of the labelled partition's cost, distortion and rate, one lane per q
      if (lane < ka.nq) {
        const int qi = lane;
        const u128 lam = (static_cast<u128>(ka.lam_hi[qi]) << 64) | ka.lam_lo[qi];
        const u128* bc = cost[qi];
        const long long o = static_cast<long long>(qi) * ka.n_regions + reg;
        u128 j = 0, d = 0;
        int bits = 0;
        if (EVN == 32) {                       // split flags, and the whole region if unsplit
          if (lab_q == 0) {
            j = lam + bc[0];
            d = edist[qi][0];
            bits = 1 + ebits[qi][0];
          } else {
            j = lam * 5u;
            bits = 5;
          }
        } else {
          j = (static_cast<u128>(ka.ev_cost[2 * o + 1]) << 64) | ka.ev_cost[2 * o];
          if (ka.ev_dist != nullptr) d = (static_cast<u128>(ka.ev_dist[2 * o + 1]) << 64) | ka.ev_dist[2 * o];
          if (ka.ev_bits != nullptr) bits = ka.ev_bits[o];
          if (lab_q != 0) {
            const int m = lab_q - 1;
            for (int q4 = 0; q4 < 4; ++q4) {
              const bool split = (m >> q4) & 1;
              if (EVN == 16 && !split) {
                j += bc[1 + q4];
                d += edist[qi][1 + q4];
                bits += ebits[qi][1 + q4];
              } else if (EVN == 8 && split) {
                const int qy = q4 >> 1, qx = q4 & 1;
                for (int dy = 0; dy < 2; ++dy)
                  for (int dx = 0; dx < 2; ++dx) {
                    const int bi = 5 + (2 * qy + dy) * 4 + 2 * qx + dx;
                    j += bc[bi];
                    d += edist[qi][bi];
                    bits += ebits[qi][bi];
                  }
              }
            }
          }
        }
        ka.ev_cost[2 * o] = static_cast<unsigned long long>(j);
        ka.ev_cost[2 * o + 1] = static_cast<unsigned long long>(j >> 64);
        if (ka.ev_dist != nullptr) {
          ka.ev_dist[2 * o] = static_cast<unsigned long long>(d);
          ka.ev_dist[2 * o + 1] = static_cast<unsigned long long>(d >> 64);
        }
        if (ka.ev_bits != nullptr) ka.ev_bits[o] = bits;
      }
      __syncwarp();
      continue;
    }
    // bottom-up choice, one lane per q (ties keep the larger transform)
    if (lane < ka.nq) {
      const int qi = lane;
      const u128 lam = (static_cast<u128>(ka.lam_hi[qi]) << 64) | ka.lam_lo[qi];
      const u128* bc = cost[qi];
      u128 j16[4], j8[4];
      int m = 0;
      u128 split = lam;
      for (int k4 = 0; k4 < 4; ++k4) {
        const int qy = k4 >> 1, qx = k4 & 1;
        j16[k4] = lam + bc[1 + k4];
        j8[k4] = lam;
        for (int dy = 0; dy < 2; ++dy)
          for (int dx = 0; dx < 2; ++dx) j8[k4] += bc[5 + (2 * qy + dy) * 4 + 2 * qx + dx];
        if (j8[k4] < j16[k4]) { m |= 1 << k4; split += j8[k4]; }
        else split += j16[k4];
      }
      const u128 whole = lam + bc[0];
      ka.labels[static_cast<long long>(qi) * ka.n_regions + reg] =
          static_cast<unsigned char>(whole <= split ? 0 : 1 + m);
      if (ka.part_cost != nullptr) {
        unsigned long long* pc = ka.part_cost + (static_cast<long long>(qi) * ka.n_regions + reg) * 34;
        pc[0] = static_cast<unsigned long long>(whole);
        pc[1] = static_cast<unsigned long long>(whole >> 64);
        for (int mm = 0; mm < 16; ++mm) {
          u128 j = lam;
          for (int k4 = 0; k4 < 4; ++k4) j += ((mm >> k4) & 1) ? j8[k4] : j16[k4];
          pc[2 + 2 * mm] = static_cast<unsigned long long>(j);
          pc[3 + 2 * mm] = static_cast<unsigned long long>(j >> 64);
        }
      }
    }
    __syncwarp();
  }
}

template <class P, typename InT, int MODE, int EVN = 0>
int launch_rd_t(const RdKernelArgs& ka, int num_sms, void* stream) {
  auto kern = rd_kernel<P, InT, MODE, EVN>;
  const size_t smem = sizeof(RdSmem) + (MODE == 2 ? sizeof(RdEvalSmem) : 0);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return static_cast<int>(e);
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kRdThreads, smem);
  if (e != cudaSuccess) return static_cast<int>(e);
  const long long work = MODE == 1 ? ka.max_count : ka.n_regions;
  const long long ctas = (work + kRdWarps - 1) / kRdWarps;
  const long long cap = static_cast<long long>(num_sms) * (occ > 0 ? occ : 1) * 8;
  const int grid = static_cast<int>(ctas < cap ? ctas : cap);
  if (grid <= 0) return 0;
  kern<<<grid, kRdThreads, smem, static_cast<cudaStream_t>(stream)>>>(ka);
  return static_cast<int>(cudaGetLastError());
}

template <int MODE, int EVN = 0>
int launch_rd_mode(int variant, int dtype, const RdKernelArgs& ka, int num_sms, void* stream) {
  if (variant == 1)
    return dtype == 0 ? launch_rd_t<ParamsTilde, uint8_t, MODE, EVN>(ka, num_sms, stream)
                      : launch_rd_t<ParamsTilde, int16_t, MODE, EVN>(ka, num_sms, stream);
  return dtype == 0 ? launch_rd_t<ParamsHat, uint8_t, MODE, EVN>(ka, num_sms, stream)
                    : launch_rd_t<ParamsHat, int16_t, MODE, EVN>(ka, num_sms, stream);
}

}  // namespace

int rd_table_words() { return 3 * 32 + 32 * 32 + 16 * 16 + 8 * 8; }

// Host tables of a variant: d_i = (T T^T)_ii per size and the fixed-point
// dequantisation scales c_ij = round(2^F sqrt(d_i / d_j)), decided exactly.
template <class P>
static void rd_tables_t(int* out) {
  int* c_out[3] = {out + 96, out + 96 + 1024, out + 96 + 1024 + 256};
  const int sizes[3] = {32, 16, 8};
  for (int z = 0; z < 3; ++z) {
    const int n = sizes[z];
    int d[32];
    for (int i = 0; i < n; ++i) d[i] = 0;
    for (int j = 0; j < n; ++j) {   // column j of T_N
      int x32[32], x16[16], x8[8];
      int* x = n == 32 ? x32 : (n == 16 ? x16 : x8);
      for (int k = 0; k < n; ++k) x[k] = (k == j);
      if (n == 32) Jam<32, P>::T(x32);
      else if (n == 16) Jam<16, P>::T(x16);
      else Jam<8, P>::T(x8);
      for (int i = 0; i < n; ++i) d[i] += x[i] * x[i];
    }
    for (int i = 0; i < 32; ++i) out[z * 32 + i] = i < n ? d[i] : 0;
    const unsigned long long lim = 1ull << (2 * (kRdFrac + 1));
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        long long c = static_cast<long long>(std::floor(std::ldexp(std::sqrt(static_cast<double>(d[i]) / d[j]),
                                                                   kRdFrac) + 0.5));
        auto ok = [&](long long cc) {   // (2cc - 1)^2 d_j <= 4^(F+1) d_i
          const unsigned long long t = static_cast<unsigned long long>(2 * cc - 1);
          return t * t * static_cast<unsigned long long>(d[j]) <= lim * static_cast<unsigned long long>(d[i]);
        };
        while (ok(c + 1)) ++c;
        while (c > 0 && !ok(c)) --c;
        c_out[z][i * n + j] = static_cast<int>(c);
      }
  }
}

void rd_tables(int variant, int* out) {
  if (variant == 1) rd_tables_t<ParamsTilde>(out);
  else rd_tables_t<ParamsHat>(out);
}

int launch_rd(int variant, int dtype, const void* in, long long pitch, long long bstride, int width, int height,
              int batch, const int* host_tables, const int* q, int nq, const unsigned long long* lam_lo,
              const unsigned long long* lam_hi, unsigned char* labels, unsigned long long* part_cost, int num_sms,
              void* stream, const RdModeArgs* mode) {
  RdKernelArgs ka;
  ka.in = in;
  ka.pitch = pitch;
  ka.bstride = bstride;
  ka.width = width;
  ka.height = height;
  ka.tiles_x = (width + 31) / 32;
  ka.tiles_per_img = ka.tiles_x * ((height + 31) / 32);
  ka.n_regions = static_cast<long long>(batch) * ka.tiles_per_img;
  ka.nq = nq;
  for (int k = 0; k < 4; ++k) {
    ka.q[k] = k < nq ? q[k] : 1;
    ka.lam_lo[k] = k < nq ? lam_lo[k] : 0;
    ka.lam_hi[k] = k < nq ? lam_hi[k] : 0;
  }
  for (int t = 0; t < rd_table_words(); ++t) ka.tables[t] = host_tables[t];
  ka.labels = labels;
  ka.part_cost = part_cost;
  ka.subset = nullptr;
  ka.subset_count = nullptr;
  ka.max_count = 0;
  ka.in_labels = nullptr;
  ka.ev_cost = nullptr;
  ka.ev_dist = nullptr;
  ka.ev_bits = nullptr;
  if (mode == nullptr || mode->mode == 0) return launch_rd_mode<0>(variant, dtype, ka, num_sms, stream);
  if (mode->mode == 1) {
    ka.subset = mode->subset;
    ka.subset_count = mode->subset_count;
    ka.max_count = mode->max_count;
    return launch_rd_mode<1>(variant, dtype, ka, num_sms, stream);
  }
  ka.in_labels = mode->in_labels;
  ka.ev_cost = mode->ev_cost;
  ka.ev_dist = mode->ev_dist;
  ka.ev_bits = mode->ev_bits;
  // one launch per size, in order: 32 initialises the outputs, 16 and 8 add to them
  int rc = launch_rd_mode<2, 32>(variant, dtype, ka, num_sms, stream);
  if (rc == 0) rc = launch_rd_mode<2, 16>(variant, dtype, ka, num_sms, stream);
  if (rc == 0) rc = launch_rd_mode<2, 8>(variant, dtype, ka, num_sms, stream);
  return rc;
}

}  // namespace cdct
