// Tensor-core (tcgen05) inference kernel of the CNN size selector.  Included
// by cnn_infer.cu inside its anonymous namespace: it uses InferArgs and the
// packed-weight layout of that file.
//
// All three convolutions run as implicit GEMMs on the 5th-generation tensor
// cores: one thread issues tcgen05.mma with bf16 operands in shared memory and
// float32 accumulators in tensor memory.  No im2col copy is made; each tap
// only moves an operand's start address.  Operands use the K-major,
// no-swizzle core-matrix layout: core matrices of 8 rows x 16 bytes, `lbo`
// bytes apart along K and `sbo` bytes apart along M (or N).
//
// conv1 and conv2 are tiled by 2 x 2 pooling WINDOWS, not by pixels: an
// accumulator row (one tensor-memory lane, one thread) holds all four pixels
// of a window as four N-groups of channels, so the max pool is three
// register maxima per channel, with no exchange between lanes.
//   conv1 (1 -> 16, 32 x 32 px): a window's receptive field is 4 x 4 input
//     pixels, exactly one K = 16 slice.  The staged region is the map
//     E[17][16] of 16-byte entries, E[j][u] = the padded pixels P[2j..2j+1]
//     [2u..2u+3] as bf16 pairs (P[2j][c], P[2j+1][c]) for c = 2u..2u+3, so
//     window (v, u) takes E[v][u] for K 0..7 and E[v+1][u] for K 8..15:
//     lbo = 256 B, sbo = 128 B.  A tile is 8 window rows (M = 128); one MMA
//     of N = 64 (window pixel g = 2 py + px, channel o) per tile, two tiles
//     per region.
//   conv2 (16 -> 32, 16 x 16 px): the windows of a PAIR of regions form the
//     M = 128 rows (core matrix i = 2 v + s: window row v of region s).  The
//     pooled conv1 maps sit in a parity-split layout, offset
//       plane * 10368 + (R & 1) * 5184 + (R >> 1) * 576 + s * 288
//       + (C & 1) * 144 + (C >> 1) * 16
//     for padded row R, column C (0..17), so that for every tap the 8
//     windows of a core matrix are 16 B apart and consecutive core matrices
//     288 B apart.  Window pixel g = (py, px) and tap (dy, dx) read the map at
//     (2 v + py + dy, 2 u + px + dx): 4 groups x 9 taps = 36 MMAs of N = 32,
//     K = 16 (lbo = a plane of 8 channels), accumulating into column group g.
//   conv3 (32 -> 32, 8 x 8 px): pixel-tiled, as its windows (2 x 16 per pair)
//     fill no tile: the pooled conv2 maps of the pair sit side by side in a
//     [4][10][20][8] map; M = 128 covers both regions, core matrix
//     k = 2 i + s (output row i of region s) at 160 k + (dy*20 + dx)*16:
//     sbo = 160 B, lbo = 3200 B; 18 MMAs (taps x channel halves), N = 32.
//     The pool is a butterfly between lanes: partners trade halves of their
//     channels and keep the maximum, twice.
// Bias and ReLU follow the maximum (both commute with it); each pooled map is
// written once, as bf16, into the next layer's map (borders stay zero).
// Weights (B operands) are repacked once per CTA into the same layout (128 B
// apart along K, 256 B along N).
//
// A CTA of 4 warps runs 16 regions per iteration, a pair at a time: both
// regions' conv1 tiles are issued together (each committed to its own
// mbarrier, so the epilogue of one tile overlaps the MMAs of the next), then
// the pair's conv2 and conv3; FC1 (warp-level MMA) and the per-slot head run
// once over the 16 regions.  The next pair's pixels are loaded into
// registers while the current pair computes.  Two CTAs share an SM.  Every
// tensor-core wait is bounded; a CTA that gives up records the error word,
// waits (bounded) for its outstanding MMAs, frees its tensor memory and stops.

constexpr int kWarpsT = 4;
constexpr int kThreadsT = 32 * kWarpsT;
constexpr int kGroupT = 16;                      // regions per CTA iteration (FC1 batch)
constexpr uint32_t kTmemColsT = 256;
// tensor-memory columns: conv1 of the pair's regions 0..127 and 128..255;
// then conv2 of the pair 0..127 and conv3 128..159
constexpr uint32_t kC1Col0 = 0, kC1Col1 = 128, kC2Col = 0, kC3Col = 128;
constexpr int kERow = 16 * 16;                   // bytes per row of the expanded map
constexpr int kEBytes = 17 * kERow;              // E[17][16] x 16 B
// conv2 input map of a pair (parity-split, see above)
constexpr int kCPar = 9 * 16;                    // one column parity of a row of a region
constexpr int kRS = 2 * kCPar;                   // a row of a region
constexpr int kRP = 2 * kRS;                     // a row of both regions
constexpr int kRPar = 9 * kRP;                   // the 9 rows of one row parity
constexpr int kA1Plane = 2 * kRPar;              // a plane of 8 channels
constexpr int kAct1T = 2 * kA1Plane;
constexpr int kA3Plane = 10 * 20 * 16;           // bytes per channel plane of the stacked conv2 map
constexpr int kAct2T = 4 * kA3Plane;             // [4][10][20][8] bf16

// shared-memory layout (bytes)
constexpr int kTCB = 0;                                     // biases b1 b2 b3 [80] float
constexpr int kTB1 = 384;                                   // conv1 B operand [64 x 16]
constexpr int kTB2 = kTB1 + 2048;                           // conv2 B operands [9 taps][1024 B]
constexpr int kTB3 = kTB2 + 9 * 1024;                       // conv3 B operands [18 slabs][1024 B]
constexpr int kTHead = kTB3 + 18 * 1024;                    // fb1, Wq, Wf2 (65-float rows), fb2
constexpr int kTE = (kTHead + kHeadBytes + 127) / 128 * 128;   // expanded maps of the pair
constexpr int kTAct1 = kTE + 2 * kEBytes;                   // conv2 input map (also the head's hidden values)
constexpr int kTAct2 = kTAct1 + kAct1T;                     // conv3 input map of the pair
constexpr int kTFeat = kTAct2 + kAct2T;                     // features [16][520] bf16
constexpr int kTU = kTFeat + kGroupT * kFeatPitch * 2;      // FC1 outputs [16][64] float
constexpr int kTLogit = kTU + kGroupT * kHidden * 4;        // logits [16][4][17] float
constexpr int kSmemT = kTLogit + kGroupT * kSlots * kLabels * 4;
static_assert(kTB1 % 128 == 0 && kTB2 % 128 == 0 && kTE % 128 == 0 && kTAct1 % 128 == 0 && kTAct2 % 128 == 0 &&
              kTFeat % 16 == 0 && kTU % 16 == 0, "alignment");
static_assert(kRP == 2 * kRS, "core matrix i = 2 v + s is kRS * i bytes from window row 0");
static_assert(kGroupT * kSlots * kHidden * 4 <= kAct1T, "the head's hidden values fit the conv2 input map");
static_assert(2 * (kSmemT + 1024) <= 228 * 1024, "two CTAs per SM");

// byte offset of padded pixel (R, C) of region s, channel plane p, in the conv2 input map
__device__ __forceinline__ int a1_off(int s, int p, int R, int C) {
  return p * kA1Plane + (R & 1) * kRPar + (R >> 1) * kRP + s * kRS + (C & 1) * kCPar + (C >> 1) * 16;
}

// B operands in the K-major core-matrix layout: element (n, k) of an N x 16
// operand at (k / 8) * 128 + (n / 8) * 256 + (n % 8) * 16 + (k % 8) * 2.
__device__ __forceinline__ int b_off(int n, int k) { return (k >> 3) * 128 + (n >> 3) * 256 + (n & 7) * 16 + (k & 7) * 2; }

//   conv1 (n, k), n = 16 g + o for window pixel g = 2 py + px, k = 8 (ry / 2) + 2 rx + ry % 2 for the
//     receptive-field pixel (ry, rx) in 0..3: W1[o][ry - py][rx - px] where both offsets are in 0..2, else 0
//   conv2 tap t: (o, c) = W2[o][t * 16 + c];  conv3 slab 2t + h: (o, c) = W3[o][t * 32 + 16 h + c]
__device__ __forceinline__ void pack_b_operands(const unsigned char* packed, unsigned char* sm, int tid) {
  const uint16_t* w1 = reinterpret_cast<const uint16_t*>(packed + kPkW1);
  const uint16_t* w2 = reinterpret_cast<const uint16_t*>(packed + kPkW2);
  const uint16_t* w3 = reinterpret_cast<const uint16_t*>(packed + kPkW3);
  for (int i = tid; i < 64 * 16; i += kThreadsT) {
    const int n = i >> 4, k = i & 15, g = n >> 4, o = n & 15;
    const int ry = 2 * (k >> 3) + (k & 1), rx = (k >> 1) & 3;
    const int dy = ry - (g >> 1), dx = rx - (g & 1);
    const bool in = dy >= 0 && dy <= 2 && dx >= 0 && dx <= 2;
    reinterpret_cast<uint16_t*>(sm + kTB1 + b_off(n, k))[0] = in ? w1[o * kW1Pitch + dy * 3 + dx] : static_cast<uint16_t>(0);
  }
  for (int i = tid; i < 9 * 32 * 16; i += kThreadsT) {
    const int t = i >> 9, o = (i >> 4) & 31, c = i & 15;
    reinterpret_cast<uint16_t*>(sm + kTB2 + t * 1024 + b_off(o, c))[0] = w2[o * kW2Pitch + t * 16 + c];
  }
  for (int i = tid; i < 18 * 32 * 16; i += kThreadsT) {
    const int sl = i >> 9, o = (i >> 4) & 31, c = i & 15;
    reinterpret_cast<uint16_t*>(sm + kTB3 + sl * 1024 + b_off(o, c))[0] =
        w3[o * kW3Pitch + (sl >> 1) * 32 + (sl & 1) * 16 + c];
  }
}

// The input rows of region `reg` that warp `warp` expands: for row pairs
// j = warp + 4k <= 16 (k < 5), the padded rows 2j and 2j + 1, i.e. input rows
// 2j - 1 and 2j (replicated beyond the image, zero outside the region), at the
// lane's column (replicated beyond the image).  Kept as raw integers and
// loaded one pair of regions ahead, so that their latency overlaps the
// previous pair's work.
template <typename InT>
__device__ __forceinline__ void load_region_rows(const InferArgs& a, long long reg, int warp, int lane, int (&px)[10]) {
  const int img = static_cast<int>(reg / a.tiles_per_img);
  const int t = static_cast<int>(reg - static_cast<long long>(img) * a.tiles_per_img);
  const int ty = t / a.tiles_x, tx = t - ty * a.tiles_x;
  const int y0 = ty * 32, x0 = tx * 32;
  const int vrows = min(32, a.height - y0), vcols = min(32, a.width - x0);
  const InT* src = static_cast<const InT*>(a.in) + img * a.bstride + x0 + min(lane, vcols - 1);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int j = warp + 4 * k;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = 2 * j - 1 + h;                       // input row of padded row 2j + h
      px[2 * k + h] = (j <= 16 && r >= 0 && r < 32) ? static_cast<int>(src[(y0 + min(r, vrows - 1)) * a.pitch]) : 0;
    }
  }
}

// The expanded map E from the loaded rows.  P = bf16(input / 64) (exact for
// |input| <= 255); the lane of input column x holds the word (P[2j][x + 1],
// P[2j + 1][x + 1]), and entry E[j][u] gathers the words of padded columns
// 2u .. 2u + 3, i.e. of lanes 2u - 1 .. 2u + 2 (zero beyond the region).
__device__ __forceinline__ void store_expanded(const int (&px)[10], unsigned char* e, int warp, int lane) {
  const int u = lane & 15;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int j = warp + 4 * k;
    if (j > 16) break;                                     // warp-uniform
    const uint32_t w = bf16_bits(static_cast<float>(px[2 * k]) * 0.015625f) |
                       (bf16_bits(static_cast<float>(px[2 * k + 1]) * 0.015625f) << 16);
    uint32_t q0 = __shfl_sync(0xffffffffu, w, (2 * u + 31) & 31), q1 = __shfl_sync(0xffffffffu, w, 2 * u);
    uint32_t q2 = __shfl_sync(0xffffffffu, w, 2 * u + 1), q3 = __shfl_sync(0xffffffffu, w, (2 * u + 2) & 31);
    if (u == 0) q0 = 0u;
    if (u == 15) q3 = 0u;
    if (lane < 16) *reinterpret_cast<uint4*>(e + j * kERow + u * 16) = make_uint4(q0, q1, q2, q3);
  }
}

// 16 float32 columns of the warp's 32 tensor-memory lanes, without waiting
// (tmem_wait_ld() before use)
__device__ __forceinline__ void tmem_ld16_nw(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// wait for this thread's tensor-memory loads; tied to the loaded registers so
// that no use of them moves above the wait
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&a)[16], uint32_t (&b)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]),
                 "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]), "+r"(a[12]), "+r"(a[13]), "+r"(a[14]), "+r"(a[15]),
                 "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7]),
                 "+r"(b[8]), "+r"(b[9]), "+r"(b[10]), "+r"(b[11]), "+r"(b[12]), "+r"(b[13]), "+r"(b[14]), "+r"(b[15])
               :
               : "memory");
}

__device__ __forceinline__ float fmax4(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  return fmaxf(fmaxf(__uint_as_float(a), __uint_as_float(b)), fmaxf(__uint_as_float(c), __uint_as_float(d)));
}

// conv1 epilogue of tile t of region s: lane l of warp w holds window
// (v, u) = (8 t + 2 w + l / 16, l % 16); its 4 x 16 columns are the window's
// pixels; the pooled pixel (16 channels) goes to padded (v + 1, u + 1).
__device__ __forceinline__ void conv1_epilogue(uint32_t taddr, unsigned char* act1, int s, int t, const float* cb,
                                               int warp, int lane) {
  uint32_t r0[16], r1[16], r2[16], r3[16];
  tmem_ld16_nw(taddr, r0);
  tmem_ld16_nw(taddr + 16, r1);
  tmem_ld16_nw(taddr + 32, r2);
  tmem_ld16_nw(taddr + 48, r3);
  tmem_wait_ld(r0, r1);
  tmem_wait_ld(r2, r3);
  uint32_t w[8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
    w[i] = pack_bf16(relu(fmax4(r0[2 * i], r1[2 * i], r2[2 * i], r3[2 * i]) + cb[2 * i]),
                     relu(fmax4(r0[2 * i + 1], r1[2 * i + 1], r2[2 * i + 1], r3[2 * i + 1]) + cb[2 * i + 1]));
  const int v = 8 * t + 2 * warp + (lane >> 4), u = lane & 15;
  unsigned char* p = act1 + a1_off(s, 0, v + 1, u + 1);
  *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
  *reinterpret_cast<uint4*>(p + kA1Plane) = make_uint4(w[4], w[5], w[6], w[7]);
}

// conv2 epilogue of the pair: lane l of warp w is M row 32 w + l = 8 i + u,
// i = 2 v + s: window (v, u) of region s; column group g = window pixel.  The
// pooled pixel (32 channels) goes to row v + 1, column 10 s + u + 1 of the
// stacked conv3 map, 8 channels per plane.
__device__ __forceinline__ void conv2_epilogue(uint32_t taddr, unsigned char* act2, const float* cb, int warp,
                                               int lane) {
  float m[32];
  {
    uint32_t a0[16], a1[16], b0[16], b1[16];
    tmem_ld16_nw(taddr, a0);
    tmem_ld16_nw(taddr + 16, a1);
    tmem_ld16_nw(taddr + 32, b0);
    tmem_ld16_nw(taddr + 48, b1);
    tmem_wait_ld(a0, a1);
    tmem_wait_ld(b0, b1);
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      m[c] = fmaxf(__uint_as_float(a0[c]), __uint_as_float(b0[c]));
      m[16 + c] = fmaxf(__uint_as_float(a1[c]), __uint_as_float(b1[c]));
    }
  }
  {
    uint32_t a0[16], a1[16], b0[16], b1[16];
    tmem_ld16_nw(taddr + 64, a0);
    tmem_ld16_nw(taddr + 80, a1);
    tmem_ld16_nw(taddr + 96, b0);
    tmem_ld16_nw(taddr + 112, b1);
    tmem_wait_ld(a0, a1);
    tmem_wait_ld(b0, b1);
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      m[c] = fmaxf(m[c], fmaxf(__uint_as_float(a0[c]), __uint_as_float(b0[c])));
      m[16 + c] = fmaxf(m[16 + c], fmaxf(__uint_as_float(a1[c]), __uint_as_float(b1[c])));
    }
  }
  const int i = 4 * warp + (lane >> 3), v = i >> 1, s = i & 1, u = lane & 7;
  const float* b = cb + 16;
  unsigned char* p = act2 + ((v + 1) * 20 + 10 * s + u + 1) * 16;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = 8 * q;
    *reinterpret_cast<uint4*>(p + q * kA3Plane) =
        make_uint4(pack_bf16(relu(m[c] + b[c]), relu(m[c + 1] + b[c + 1])),
                   pack_bf16(relu(m[c + 2] + b[c + 2]), relu(m[c + 3] + b[c + 3])),
                   pack_bf16(relu(m[c + 4] + b[c + 4]), relu(m[c + 5] + b[c + 5])),
                   pack_bf16(relu(m[c + 6] + b[c + 6]), relu(m[c + 7] + b[c + 7])));
  }
}

// conv3 epilogue of a pair: lane l of warp w holds core matrix k = 4w + l / 8
// (region s = k & 1, output row i = k >> 1), column l % 8; the y neighbour is
// 16 lanes away.  Butterfly pool: partners (lane ^ 1, then lane ^ 16) trade
// halves of their channels and keep the maximum, so each lane of a window ends
// with channels 8 q .. 8 q + 7, q = 2 (lane & 1) + (lane >> 4 & 1).  Pooled
// pixel (py = w, px) of region s goes to the region's feature row at
// (py * 4 + px) * 32 + 8 q.
__device__ __forceinline__ void conv3_epilogue(uint32_t taddr, unsigned char* feat_pair, const float* cb, int warp,
                                               int lane) {
  uint32_t lo[16], hi[16];
  tmem_ld16_nw(taddr, lo);
  tmem_ld16_nw(taddr + 16, hi);
  tmem_wait_ld(lo, hi);
  const bool xo = lane & 1, yo = (lane & 16) != 0;
  float v[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const float a = __uint_as_float(lo[c]), b = __uint_as_float(hi[c]);
    v[c] = fmaxf(xo ? b : a, __shfl_xor_sync(0xffffffffu, xo ? a : b, 1));
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) v[c] = fmaxf(yo ? v[8 + c] : v[c], __shfl_xor_sync(0xffffffffu, yo ? v[c] : v[8 + c], 16));
  const int q = 2 * (lane & 1) + ((lane >> 4) & 1);
  const int s = (lane >> 3) & 1, px = (lane & 7) >> 1, py = warp;
  const float* b = cb + 48 + 8 * q;
  *reinterpret_cast<uint4*>(feat_pair + s * kFeatPitch * 2 + ((py * 4 + px) * 32 + 8 * q) * 2) =
      make_uint4(pack_bf16(relu(v[0] + b[0]), relu(v[1] + b[1])), pack_bf16(relu(v[2] + b[2]), relu(v[3] + b[3])),
                 pack_bf16(relu(v[4] + b[4]), relu(v[5] + b[5])), pack_bf16(relu(v[6] + b[6]), relu(v[7] + b[7])));
}

// the region that CTA position `idx` (0 .. kGroupT) of the group at `base`
// computes; the position kGroupT is the next group's first.  A region past
// the end is clamped: computed, never written out.
__device__ __forceinline__ long long infer_region(const InferArgs& a, long long base, long long stride, int idx) {
  const long long r = idx < kGroupT ? base + idx : base + stride + (idx - kGroupT);
  return r < a.n_regions ? r : a.n_regions - 1;
}

template <typename InT>
__global__ void __launch_bounds__(kThreadsT, 2) cnn_infer_tc_kernel(const InferArgs a, int* __restrict__ err,
                                                                     long long wait_limit) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar1[4];   // conv1 tiles (region, tile) of the pair
  __shared__ __align__(8) uint64_t bar2;      // conv2 of the pair
  __shared__ __align__(8) uint64_t bar3;      // conv3 of the pair
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  {
    const float* cbs = reinterpret_cast<const float*>(a.packed + kPkCB);
    for (int i = tid; i < 80; i += kThreadsT) reinterpret_cast<float*>(sm + kTCB)[i] = cbs[i];
    const float* hs = reinterpret_cast<const float*>(a.packed + kPkHead);
    float* hd = reinterpret_cast<float*>(sm + kTHead);
    constexpr int nq = kHidden + kHidden * kSlots;
    for (int i = tid; i < nq; i += kThreadsT) hd[i] = hs[i];
    for (int i = tid; i < kLabels * kHidden; i += kThreadsT) hd[nq + (i / kHidden) * kF2Pitch + i % kHidden] = hs[nq + i];
    for (int i = tid; i < kLabels; i += kThreadsT) hd[nq + kLabels * kF2Pitch + i] = hs[nq + kLabels * kHidden + i];
    pack_b_operands(a.packed, sm, tid);
    // zero both activation maps (borders stay zero; interiors are rewritten)
    for (int i = tid; i < (kTFeat - kTAct1) / 16; i += kThreadsT)
      reinterpret_cast<uint4*>(sm + kTAct1)[i] = make_uint4(0, 0, 0, 0);
  }
  if (warp == 0) tmem_alloc(&tmem_base, kTmemColsT);
  if (tid == 0) {
    for (int j = 0; j < 4; ++j) mbar_init(&bar1[j], 1);
    mbar_init(&bar2, 1);
    mbar_init(&bar3, 1);
    fence_mbar_init();
  }
  fence_proxy_async_smem();                   // B operands and zeroed maps are read by the tensor cores
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  const float* cb = reinterpret_cast<const float*>(sm + kTCB);
  unsigned char* feat = sm + kTFeat;
  unsigned char* act1 = sm + kTAct1;
  unsigned char* act2 = sm + kTAct2;
  float* u_s = reinterpret_cast<float*>(sm + kTU);
  float* logit_s = reinterpret_cast<float*>(sm + kTLogit);
  float* g_s = reinterpret_cast<float*>(sm + kTAct1);       // the head's hidden values (the map is free then)
  const float* fb1 = reinterpret_cast<const float*>(sm + kTHead);
  const float* wq = fb1 + kHidden;
  const float* wf2 = wq + kHidden * kSlots;
  const float* fb2 = wf2 + kLabels * kF2Pitch;
  const int ns = a.n_slots;
  constexpr uint32_t idesc64 = idesc_bf16_f32(128, 64), idesc32 = idesc_bf16_f32(128, 32);
  const uint32_t e_s = smem_u32(sm + kTE), act1_s = smem_u32(act1), act2_s = smem_u32(act2);
  const uint32_t b1_s = smem_u32(sm + kTB1), b2_s = smem_u32(sm + kTB2), b3_s = smem_u32(sm + kTB3);
  const uint32_t wl = static_cast<uint32_t>(warp * 32) << 16;   // the warp's tensor-memory lanes
  const long long stride = static_cast<long long>(gridDim.x) * kGroupT;
  uint32_t ph = 0;
  bool ok = true, failed = false;
  int px0[10], px1[10];
  {
    const long long base0 = static_cast<long long>(blockIdx.x) * kGroupT;
    load_region_rows<InT>(a, infer_region(a, base0, stride, 0), warp, lane, px0);
    load_region_rows<InT>(a, infer_region(a, base0, stride, 1), warp, lane, px1);
  }

  for (long long base = static_cast<long long>(blockIdx.x) * kGroupT; base < a.n_regions && !failed; base += stride) {
#pragma unroll 1
    for (int pr = 0; pr < kGroupT / 2 && !failed; ++pr) {
      store_expanded(px0, sm + kTE, warp, lane);
      store_expanded(px1, sm + kTE + kEBytes, warp, lane);
      fence_proxy_async_smem();               // the expanded maps are read by the tensor cores
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      // conv1: tile (s, t) = window rows 8 t .. 8 t + 7 of region s, one MMA of K = 16, N = 64
      if (tid == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int s = q >> 1, tt = q & 1;
          umma_bf16(tmem + (s ? kC1Col1 : kC1Col0) + 64 * tt,
                    umma_desc(e_s + s * kEBytes + tt * 8 * kERow, kERow, 128), umma_desc(b1_s, 128, 256), idesc64, 0u);
          umma_commit(&bar1[q]);
        }
      }
      load_region_rows<InT>(a, infer_region(a, base, stride, 2 * pr + 2), warp, lane, px0);
      load_region_rows<InT>(a, infer_region(a, base, stride, 2 * pr + 3), warp, lane, px1);
#pragma unroll 1
      for (int q = 0; q < 4; ++q) {
        ok &= mbar_wait_bounded(&bar1[q], ph, wait_limit);
        tc_fence_after();
        const int s = q >> 1, tt = q & 1;
        conv1_epilogue(tmem + wl + (s ? kC1Col1 : kC1Col0) + 64 * tt, act1, s, tt, cb, warp, lane);
      }
      fence_proxy_async_smem();               // the conv2 input map is read by the tensor cores
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      // conv2 of the pair: window pixel gp = (py, px) x tap (dy, dx), K = 16 over 2 planes, N = 32
      if (tid == 0) {
#pragma unroll
        for (int gp = 0; gp < 4; ++gp) {
#pragma unroll
          for (int tap = 0; tap < 9; ++tap) {
            const int ry = (gp >> 1) + tap / 3, rx = (gp & 1) + tap % 3;
            const uint32_t ab = act1_s + (ry & 1) * kRPar + (ry >> 1) * kRP + (rx & 1) * kCPar + (rx >> 1) * 16;
            umma_bf16(tmem + kC2Col + 32 * gp, umma_desc(ab, kA1Plane, kRS), umma_desc(b2_s + tap * 1024, 128, 256),
                      idesc32, tap > 0 ? 1u : 0u);
          }
        }
        umma_commit(&bar2);
      }
      ok &= mbar_wait_bounded(&bar2, ph, wait_limit);
      tc_fence_after();
      conv2_epilogue(tmem + wl + kC2Col, act2, cb, warp, lane);
      fence_proxy_async_smem();               // the stacked conv3 map is read by the tensor cores
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      // conv3 of the pair: 9 taps x 2 channel halves of K = 16, N = 32
      if (tid == 0) {
#pragma unroll
        for (int k = 0; k < 18; ++k) {
          const int tap = k >> 1, h = k & 1;
          umma_bf16(tmem + kC3Col, umma_desc(act2_s + ((tap / 3) * 20 + tap % 3) * 16 + 2 * h * kA3Plane, kA3Plane, 160),
                    umma_desc(b3_s + k * 1024, 128, 256), idesc32, k > 0 ? 1u : 0u);
        }
        umma_commit(&bar3);
      }
      ok &= mbar_wait_bounded(&bar3, ph, wait_limit);
      tc_fence_after();
      conv3_epilogue(tmem + wl + kC3Col, feat + (2 * pr) * kFeatPitch * 2, cb, warp, lane);
      ph ^= 1u;
      tc_fence_before();
      failed = !__syncthreads_and(ok);        // features written; tensor memory and maps free again
      tc_fence_after();
    }
    if (failed) break;
    // FC1: u[16 regions][64] = features x Wf1^T (warp-level MMA); warp = neuron tile of 16
    {
      const int mt = warp;
      const uint4* f1 = reinterpret_cast<const uint4*>(a.packed + kPkF1) + mt * 32 * 32 + lane;
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const uint32_t b_lane = smem_u32(feat) + ((nt * 8 + (lane & 7)) * kFeatPitch + (lane >> 3) * 8) * 2;
#pragma unroll 4
        for (int ks = 0; ks < 32; ks += 2) {
          uint32_t bb[4];
          ldsm_x4(bb, b_lane + ks * 32);
          const uint4 a0 = __ldg(f1 + ks * 32), a1 = __ldg(f1 + (ks + 1) * 32);
          const uint32_t af0[4] = {a0.x, a0.y, a0.z, a0.w}, af1[4] = {a1.x, a1.y, a1.z, a1.w};
          const uint32_t b0[2] = {bb[0], bb[1]}, b1[2] = {bb[2], bb[3]};
          mma_bf16(acc, af0, b0);
          mma_bf16(acc, af1, b1);
        }
        const int n0 = mt * 16 + g, r0 = nt * 8 + 2 * t;
        u_s[r0 * kHidden + n0] = acc[0];
        u_s[(r0 + 1) * kHidden + n0] = acc[1];
        u_s[r0 * kHidden + n0 + 8] = acc[2];
        u_s[(r0 + 1) * kHidden + n0 + 8] = acc[3];
      }
    }
    __syncthreads();
    // head, once per (region, slot): g = bf16(relu(u + fb1 + Wq[:, slot])); then
    // logits[region][slot][label] = fb2 + Wf2 g
    for (int i = tid; i < kGroupT * ns * kHidden; i += kThreadsT) {
      const int h = i % kHidden, rs = i / kHidden, si = rs % ns, region = rs / ns;
      g_s[(region * kSlots + si) * kHidden + h] =
          round_bf16(relu((u_s[region * kHidden + h] + fb1[h]) + wq[h * kSlots + a.slots[si]]));
    }
    __syncthreads();
    {
      const int per = ns * kLabels;
      for (int task = tid; task < kGroupT * per; task += kThreadsT) {
        const int region = task / per, rem = task - region * per;
        const int si = rem / kLabels, j = rem - si * kLabels;
        const float* gv = g_s + (region * kSlots + si) * kHidden;
        const float* w = wf2 + j * kF2Pitch;
        float acc = fb2[j];
#pragma unroll 8
        for (int h = 0; h < kHidden; ++h) acc = fmaf(w[h], gv[h], acc);
        logit_s[(region * kSlots + si) * kLabels + j] = acc;
      }
    }
    __syncthreads();
    if (tid < kGroupT * ns) {
      const int region = tid / ns, si = tid - region * ns;
      const long long reg = base + region;
      if (reg < a.n_regions) {
        const float* l = logit_s + (region * kSlots + si) * kLabels;
        int best = 0;
        float b1 = l[0], b2 = -INFINITY;
        for (int j = 1; j < kLabels; ++j) {
          if (l[j] > b1) { b2 = b1; b1 = l[j]; best = j; }
          else if (l[j] > b2) b2 = l[j];
        }
        const long long o = static_cast<long long>(si) * a.n_regions + reg;
        a.labels[o] = static_cast<unsigned char>(best);
        if (a.margin != nullptr) a.margin[o] = b1 - b2;
        if (a.logits != nullptr)
          for (int j = 0; j < kLabels; ++j) a.logits[o * kLabels + j] = l[j];
      }
    }
    // the head's hidden values used the conv2 input map: clear it (its borders
    // must be zero) before the next group's first pair
    __syncthreads();
    for (int i = tid; i < kAct1T / 16; i += kThreadsT) reinterpret_cast<uint4*>(sm + kTAct1)[i] = make_uint4(0, 0, 0, 0);
    fence_proxy_async_smem();
    __syncthreads();
  }
  if (failed && tid == 0) {
    atomicOr(err, 2);
    // the MMAs that may still run: each barrier's last armed phase
    for (int j = 0; j < 4; ++j) (void)mbar_wait_bounded(&bar1[j], ph ^ 1u, wait_limit);
    (void)mbar_wait_bounded(&bar2, ph ^ 1u, wait_limit);
    (void)mbar_wait_bounded(&bar3, ph ^ 1u, wait_limit);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemColsT);
}

template <typename InT>
int launch_infer_tc_t(const InferArgs& a, int num_sms, int* err, void* stream) {
  auto kern = cnn_infer_tc_kernel<InT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemT);
  if (e != cudaSuccess) return static_cast<int>(e);
  const long long groups = (a.n_regions + kGroupT - 1) / kGroupT;
  const long long cap = 2ll * num_sms;
  const int grid = static_cast<int>(groups < cap ? groups : cap);
  if (grid <= 0) return 0;
  long long limit = kDefaultWaitLimit;
  (void)fault_mode(&limit);
  kern<<<grid, kThreadsT, kSmemT, static_cast<cudaStream_t>(stream)>>>(a, err, limit);
  return static_cast<int>(cudaGetLastError());
}
