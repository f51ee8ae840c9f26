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
//     288 B apart.  A window's receptive field is 4 x 4 pixels: one MMA per
//     offset (ry, rx) in it reads the map at (2 v + ry, 2 u + rx) with K = 16
//     (lbo = a plane of 8 channels) and N = 128 = window pixel g x 32
//     channels, whose B operand holds W2's tap (ry - py, rx - px) for pixel g
//     = (py, px), or zeros where that is not a tap: 16 MMAs per pair.
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
// One CTA per SM (all 512 tensor-memory columns), warp-specialised, runs a
// software pipeline over pairs of regions:
//   2 staging warps load pair k + 1's pixels while expanding pair k into one
//     of two expanded-map slots;
//   1 MMA warp issues, in iteration k, conv1 of pair k, conv2 of pair k - 1
//     and conv3 of pair k - 2 (activation maps double-buffered), each as soon
//     as its inputs are written and its accumulators drained;
//   8 epilogue warps drain the accumulators in completion order (warps w and
//     w + 4 read the same tensor-memory lanes and split the channels) and run
//     FC1 and the per-slot head every 8 pairs.
// The roles meet on mbarriers only.  The tensor core's cost here is set by
// the A operand: an M = 128, K = 16 MMA reads 4 KB of shared memory whatever
// N is (up to 128), which is why conv2 uses N = 128.  Every wait is bounded;
// a role that gives up raises a shared abort flag that ends the others' waits,
// the MMA warp waits (bounded) for its outstanding MMAs, and the CTA records
// the error word and frees its tensor memory.

constexpr int kWarpsT = 8;                       // epilogue warps (two per tensor-memory lane quadrant)
constexpr int kThreadsT = 32 * kWarpsT;
constexpr int kIssuerWarp = kWarpsT, kProducerWarp0 = kWarpsT + 1, kProducerWarps = 2;
constexpr int kBlockT = kThreadsT + 32 * (1 + kProducerWarps);   // + the MMA-issuing warp and the staging warps
constexpr int kGroupT = 16;                      // regions per FC1 batch
constexpr int kPairsT = kGroupT / 2;
constexpr uint32_t kTmemColsT = 512;
// tensor-memory columns: conv1 of a pair (4 tiles of 64), conv2 of a pair, conv3 of a pair
constexpr uint32_t kC1Col = 0, kC2Col = 256, kC3Col = 384;
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

// shared-memory layout (bytes); the activation maps are double-buffered
constexpr int kTCB = 0;                                     // biases b1 b2 b3 [80] float
constexpr int kTB1 = 384;                                   // conv1 B operand [64 x 16]
constexpr int kTB2 = kTB1 + 2048;                           // conv2 B operands [16 offsets][4096 B]
constexpr int kTB3 = kTB2 + 16 * 4096;                      // conv3 B operands [18 slabs][1024 B]
constexpr int kTHead = kTB3 + 18 * 1024;                    // fb1, Wq, Wf2 (68-float rows), fb2
constexpr int kTE = (kTHead + kHeadBytes + 127) / 128 * 128;   // expanded maps [2 slots][2 regions]
constexpr int kTAct1 = kTE + 4 * kEBytes;                   // conv2 input maps [2]
constexpr int kTAct2 = kTAct1 + 2 * kAct1T;                 // conv3 input maps [2]
constexpr int kTFeat = kTAct2 + 2 * kAct2T;                 // features [16][520] bf16
constexpr int kHPitch = kHidden + 8;                        // bf16 per row of the hidden values and of Wf2
constexpr int kTU = kTFeat + kGroupT * kFeatPitch * 2;      // FC1 partial outputs [2 K halves][16][64] float
constexpr int kTG = kTU + 2 * kGroupT * kHidden * 4;        // hidden values [16 regions x 4 slots][72] bf16
constexpr int kTW2 = kTG + kGroupT * kSlots * kHPitch * 2;  // Wf2 [24 labels (17 + zero rows)][72] bf16
constexpr int kTLogit = kTW2 + 24 * kHPitch * 2;            // logits [16][4][17] float
constexpr int kSmemT = kTLogit + kGroupT * kSlots * kLabels * 4;
static_assert(kTB1 % 128 == 0 && kTB2 % 128 == 0 && kTE % 128 == 0 && kTAct1 % 128 == 0 && kTAct2 % 128 == 0 &&
              kTFeat % 16 == 0 && kTU % 16 == 0 && kTG % 16 == 0 && kTW2 % 16 == 0, "alignment");
static_assert(kRP == 2 * kRS, "core matrix i = 2 v + s is kRS * i bytes from window row 0");
static_assert(kSmemT + 1024 <= 227 * 1024, "one CTA per SM");

// byte offset of padded pixel (R, C) of region s, channel plane p, in the conv2 input map
__device__ __forceinline__ int a1_off(int s, int p, int R, int C) {
  return p * kA1Plane + (R & 1) * kRPar + (R >> 1) * kRP + s * kRS + (C & 1) * kCPar + (C >> 1) * 16;
}

// B operands in the K-major core-matrix layout: element (n, k) of an N x 16
// operand at (k / 8) * 128 + (n / 8) * 256 + (n % 8) * 16 + (k % 8) * 2.
__device__ __forceinline__ int b_off(int n, int k) { return (k >> 3) * 128 + (n >> 3) * 256 + (n & 7) * 16 + (k & 7) * 2; }

//   conv1 (n, k), n = 16 g + o for window pixel g = 2 py + px, k = 8 (ry / 2) + 2 rx + ry % 2 for the
//     receptive-field pixel (ry, rx) in 0..3: W1[o][ry - py][rx - px] where both offsets are in 0..2, else 0
//   conv2 offset (ry, rx) in 0..3: (n, c), n = 32 g + o for window pixel g = 2 py + px:
//     W2[o][((ry - py) * 3 + rx - px) * 16 + c] where both offsets are in 0..2, else 0
//   conv3 slab 2t + h: (o, c) = W3[o][t * 32 + 16 h + c]
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
  for (int i = tid; i < 16 * 128 * 16; i += kThreadsT) {
    const int off = i >> 11, n = (i >> 4) & 127, c = i & 15, g = n >> 5, o = n & 31;
    const int dy = (off >> 2) - (g >> 1), dx = (off & 3) - (g & 1);
    const bool in = dy >= 0 && dy <= 2 && dx >= 0 && dx <= 2;
    reinterpret_cast<uint16_t*>(sm + kTB2 + off * 4096 + b_off(n, c))[0] =
        in ? w2[o * kW2Pitch + (dy * 3 + dx) * 16 + c] : static_cast<uint16_t>(0);
  }
  for (int i = tid; i < 18 * 32 * 16; i += kThreadsT) {
    const int sl = i >> 9, o = (i >> 4) & 31, c = i & 15;
    reinterpret_cast<uint16_t*>(sm + kTB3 + sl * 1024 + b_off(o, c))[0] =
        w3[o * kW3Pitch + (sl >> 1) * 32 + (sl & 1) * 16 + c];
  }
}

// Staging: a warp per region of the pair expands rows j of its expanded map,
// half 0 (j in [0, 9)) and half 1 (j in [9, 17)), from input
// rows 2j - 1 and 2j (17 and 16 rows; replicated beyond the image, zero
// outside the region) at the lane's column (replicated beyond the image).
// The pixels are kept as raw integers and loaded one pair of regions ahead.
constexpr int kStageRows = 17;
template <typename InT>
__device__ __forceinline__ void load_half_region(const InferArgs& a, long long reg, int half, int lane,
                                                 int (&px)[kStageRows]) {
  const unsigned r32 = static_cast<unsigned>(reg);          // below 2^31 (checked by the caller)
  const unsigned img = r32 / static_cast<unsigned>(a.tiles_per_img);
  const unsigned t = r32 - img * static_cast<unsigned>(a.tiles_per_img);
  const int ty = static_cast<int>(t / static_cast<unsigned>(a.tiles_x)), tx = static_cast<int>(t) - ty * a.tiles_x;
  const int y0 = ty * 32, x0 = tx * 32;
  const int vrows = min(32, a.height - y0), vcols = min(32, a.width - x0);
  const InT* src = static_cast<const InT*>(a.in) + static_cast<long long>(img) * a.bstride + x0 + min(lane, vcols - 1);
  // half 0: input rows 0..16 (j = 0..8 use rows -1..16); half 1: rows 17..31 (j = 9..16 use rows 17..32)
  const int r0 = half ? 17 : 0, nr = half ? 15 : 17;
#pragma unroll
  for (int i = 0; i < kStageRows; ++i)
    px[i] = i < nr ? static_cast<int>(src[(y0 + min(r0 + i, vrows - 1)) * a.pitch]) : 0;
}

// Rows j of the expanded map E of a region from the loaded pixels (half 0:
// j = 0..8; half 1: j = 9..16).  P = bf16(input / 64) (exact for |input| <=
// 255) with a zero border; the lane of input column x forms the word
// (P[2j][x + 1], P[2j + 1][x + 1]) = (input row 2j - 1, row 2j), and entry
// E[j][u] gathers the words of padded columns 2u .. 2u + 3, i.e. of lanes
// 2u - 1 .. 2u + 2 (zero beyond the region).
__device__ __forceinline__ void store_half_expanded(const int (&px)[kStageRows], int half, unsigned char* e, int lane) {
  const int u = lane & 15;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    if (half && i == 8) break;
    const int j = half ? 9 + i : i;
    // input row 2j - 1 is px[2j - 1 - r0], row 2j is px[2j - r0] (r0 = 0 or 17)
    const int lo_i = half ? 2 * i : 2 * i - 1, hi_i = half ? 2 * i + 1 : 2 * i;
    const float lo = lo_i >= 0 ? static_cast<float>(px[lo_i]) : 0.f;
    const float hi = (half && i == 7) ? 0.f : static_cast<float>(px[hi_i]);
    const uint32_t w = bf16_bits(lo * 0.015625f) | (bf16_bits(hi * 0.015625f) << 16);
    uint32_t q0 = __shfl_sync(0xffffffffu, w, (2 * u + 31) & 31), q1 = __shfl_sync(0xffffffffu, w, 2 * u);
    uint32_t q2 = __shfl_sync(0xffffffffu, w, 2 * u + 1), q3 = __shfl_sync(0xffffffffu, w, (2 * u + 2) & 31);
    if (u == 0) q0 = 0u;
    if (u == 15) q3 = 0u;
    if (lane < 16) *reinterpret_cast<uint4*>(e + j * kERow + u * 16) = make_uint4(q0, q1, q2, q3);
  }
}

// 8 float32 columns of the warp's 32 tensor-memory lanes, without waiting
__device__ __forceinline__ void tmem_ld8_nw(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
// wait for this thread's tensor-memory loads; tied to the loaded registers so
// that no use of them moves above the wait
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&a)[8], uint32_t (&b)[8], uint32_t (&c)[8], uint32_t (&d)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]),
                 "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7]),
                 "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3]), "+r"(c[4]), "+r"(c[5]), "+r"(c[6]), "+r"(c[7]),
                 "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3]), "+r"(d[4]), "+r"(d[5]), "+r"(d[6]), "+r"(d[7])
               :
               : "memory");
}

__device__ __forceinline__ float fmax4(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  return fmaxf(fmaxf(__uint_as_float(a), __uint_as_float(b)), fmaxf(__uint_as_float(c), __uint_as_float(d)));
}
__device__ __forceinline__ uint32_t pack_relu_bias(float x, float y, const float* b) {
  return pack_bf16(relu(x + b[0]), relu(y + b[1]));
}

// The two warps w and w + 4 read the same tensor-memory lanes (lane quadrant
// w % 4) and split the channels: warp half h = w / 4 takes the upper or lower
// half of them.

// conv1 epilogue of the pair (all four tiles loaded before one wait): tile
// q = 2 s + t, lane l of quadrant wq holds window (v, u) = (8 t + 2 wq + l / 16,
// l % 16) of region s; its 4 x 16 columns are the window's pixels; the pooled
// channels 8 h .. 8 h + 7 go to plane h at padded (v + 1, u + 1).
__device__ __forceinline__ void conv1_epilogue(uint32_t taddr, unsigned char* act1, const float* cb, int warp,
                                               int lane) {
  const int h = warp >> 2, wq = warp & 3;
  uint32_t r[4][4][8];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int gp = 0; gp < 4; ++gp) tmem_ld8_nw(taddr + 64 * q + 16 * gp + 8 * h, r[q][gp]);
#pragma unroll
  for (int q = 0; q < 4; ++q) tmem_wait_ld(r[q][0], r[q][1], r[q][2], r[q][3]);
  const float* b = cb + 8 * h;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
      w[i] = pack_relu_bias(fmax4(r[q][0][2 * i], r[q][1][2 * i], r[q][2][2 * i], r[q][3][2 * i]),
                            fmax4(r[q][0][2 * i + 1], r[q][1][2 * i + 1], r[q][2][2 * i + 1], r[q][3][2 * i + 1]),
                            b + 2 * i);
    const int v = 8 * (q & 1) + 2 * wq + (lane >> 4), u = lane & 15;
    *reinterpret_cast<uint4*>(act1 + a1_off(q >> 1, h, v + 1, u + 1)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// conv2 epilogue of the pair: lane l of quadrant wq is M row 32 wq + l =
// 8 i + u, i = 2 v + s: window (v, u) of region s; column group g (32 columns)
// = window pixel.  The pooled channels 16 h .. 16 h + 15 go to planes 2 h and
// 2 h + 1 at row v + 1, column 10 s + u + 1 of the stacked conv3 map.
__device__ __forceinline__ void conv2_epilogue(uint32_t taddr, unsigned char* act2, const float* cb, int warp,
                                               int lane) {
  const int h = warp >> 2, wq = warp & 3;
  const int i = 4 * wq + (lane >> 3), v = i >> 1, s = i & 1, u = lane & 7;
  unsigned char* p = act2 + ((v + 1) * 20 + 10 * s + u + 1) * 16;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int c0 = 16 * h + 8 * e;
    uint32_t r0[8], r1[8], r2[8], r3[8];
    tmem_ld8_nw(taddr + c0, r0);
    tmem_ld8_nw(taddr + 32 + c0, r1);
    tmem_ld8_nw(taddr + 64 + c0, r2);
    tmem_ld8_nw(taddr + 96 + c0, r3);
    tmem_wait_ld(r0, r1, r2, r3);
    const float* b = cb + 16 + c0;
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      w[k] = pack_relu_bias(fmax4(r0[2 * k], r1[2 * k], r2[2 * k], r3[2 * k]),
                            fmax4(r0[2 * k + 1], r1[2 * k + 1], r2[2 * k + 1], r3[2 * k + 1]), b + 2 * k);
    *reinterpret_cast<uint4*>(p + (2 * h + e) * kA3Plane) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// conv3 epilogue of a pair: lane l of quadrant wq holds core matrix k = 4 wq + l / 8 (region s = k & 1, output row i = k >> 1), column l % 8; the
// y neighbour is 16 lanes away.  Butterfly pool over the warp's 16 channels
// 16 h ..: partners (lane ^ 1, then lane ^ 16) trade halves and keep the
// maximum, so each lane of a window ends with channels 16 h + 4 q .. + 3,
// q = 2 (lane & 1) + (lane >> 4 & 1).  Pooled pixel (py = wq, px) of region s
// goes to the region's feature row at (py * 4 + px) * 32 + 16 h + 4 q.
__device__ __forceinline__ void conv3_epilogue(uint32_t taddr, unsigned char* feat_pair, const float* cb, int warp,
                                               int lane) {
  const int h = warp >> 2, wq = warp & 3;
  uint32_t lo[8], hi[8], unused0[8], unused1[8];
  tmem_ld8_nw(taddr + 16 * h, lo);
  tmem_ld8_nw(taddr + 16 * h + 8, hi);
  tmem_wait_ld(lo, hi, unused0, unused1);
  const bool xo = lane & 1, yo = (lane & 16) != 0;
  float v[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float a = __uint_as_float(lo[c]), b = __uint_as_float(hi[c]);
    v[c] = fmaxf(xo ? b : a, __shfl_xor_sync(0xffffffffu, xo ? a : b, 1));
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) v[c] = fmaxf(yo ? v[4 + c] : v[c], __shfl_xor_sync(0xffffffffu, yo ? v[c] : v[4 + c], 16));
  const int q = 2 * (lane & 1) + ((lane >> 4) & 1);
  const int s = (lane >> 3) & 1, px = (lane & 7) >> 1, py = wq;
  const float* b = cb + 48 + 16 * h + 4 * q;
  *reinterpret_cast<uint2*>(feat_pair + s * kFeatPitch * 2 + ((py * 4 + px) * 32 + 16 * h + 4 * q) * 2) =
      make_uint2(pack_relu_bias(v[0], v[1], b), pack_relu_bias(v[2], v[3], b + 2));
}

// Region s (0, 1) of pair k of this CTA: pairs run through the CTA's groups
// of 16 regions (group n at blockIdx.x * 16 + n * stride), 8 pairs a group.
// A region past the end is clamped: computed, never written out.
__device__ __forceinline__ long long pair_region(const InferArgs& a, long long k, int s) {
  const long long n = k / kPairsT;
  const long long r = (static_cast<long long>(blockIdx.x) + n * gridDim.x) * kGroupT + 2 * (k - n * kPairsT) + s;
  return r < a.n_regions ? r : a.n_regions - 1;
}

// barrier among the epilogue warps only (hardware barrier 1)
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kThreadsT) : "memory"); }
// the same, returning whether `pred` holds in every epilogue thread
__device__ __forceinline__ bool epi_sync_and(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.and.pred p, 1, %2, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"(static_cast<uint32_t>(pred)), "n"(kThreadsT)
      : "memory");
  return r != 0;
}

// Wait for phase `parity` of `bar`; false once the CTA has given up (the
// shared flag `abort`) or after about `limit` SM cycles, which also sets the flag.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, long long limit, volatile int* abort) {
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

// FC1 and the per-slot head of the group at `base` (epilogue warps; features complete)
//   u = Wf1 f (FC1; warp (mt, kh) = neuron tile of 16 x half of K, both region tiles, so that each
//       Wf1 fragment is read once; the two K halves are added in a fixed order)
//   g = bf16(relu(u + fb1 + Wq[:, slot]))  per (region, slot): rows region * 4 + slot
//   logits = g Wf2^T + fb2  (warp-level MMA: 4 row tiles x 3 label tiles of 8, K = 64)
//   label = the first maximum, margin = best minus second best
__device__ __forceinline__ void group_head(const InferArgs& a, long long base, unsigned char* sm, int tid) {
  const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const unsigned char* feat = sm + kTFeat;
  float* u_s = reinterpret_cast<float*>(sm + kTU);
  uint16_t* g_s = reinterpret_cast<uint16_t*>(sm + kTG);
  float* logit_s = reinterpret_cast<float*>(sm + kTLogit);
  const float* fb1 = reinterpret_cast<const float*>(sm + kTHead);
  const float* wq = fb1 + kHidden;
  const float* fb2 = wq + kHidden * kSlots + kLabels * kF2Pitch;
  const int ns = a.n_slots;
  {
    const int mt = warp & 3, kh = warp >> 2;
    const uint4* f1 = reinterpret_cast<const uint4*>(a.packed + kPkF1) + mt * 32 * 32 + lane;
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    const uint32_t b_lane = smem_u32(feat) + ((lane & 7) * kFeatPitch + (lane >> 3) * 8) * 2;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int ks = 16 * kh + 2 * i;
      const uint4 a0 = __ldg(f1 + ks * 32), a1 = __ldg(f1 + (ks + 1) * 32);
      const uint32_t af0[4] = {a0.x, a0.y, a0.z, a0.w}, af1[4] = {a1.x, a1.y, a1.z, a1.w};
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        uint32_t bb[4];
        ldsm_x4(bb, b_lane + nt * 8 * kFeatPitch * 2 + ks * 32);
        const uint32_t b0[2] = {bb[0], bb[1]}, b1[2] = {bb[2], bb[3]};
        mma_bf16(acc[nt], af0, b0);
        mma_bf16(acc[nt], af1, b1);
      }
    }
    float* up = u_s + kh * kGroupT * kHidden;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const int n0 = mt * 16 + g, r0 = nt * 8 + 2 * t;
      up[r0 * kHidden + n0] = acc[nt][0];
      up[(r0 + 1) * kHidden + n0] = acc[nt][1];
      up[r0 * kHidden + n0 + 8] = acc[nt][2];
      up[(r0 + 1) * kHidden + n0 + 8] = acc[nt][3];
    }
  }
  epi_sync();
  for (int i = tid; i < kGroupT * kHidden; i += kThreadsT) {
    const int h = i % kHidden, region = i / kHidden;
    const float uh = (u_s[i] + u_s[kGroupT * kHidden + i]) + fb1[h];
#pragma unroll
    for (int si = 0; si < kSlots; ++si)
      if (si < ns) g_s[(region * kSlots + si) * kHPitch + h] = static_cast<uint16_t>(bf16_bits(relu(uh + wq[h * kSlots + a.slots[si]])));
  }
  epi_sync();
  {
    const int mt = warp & 3;
    const uint32_t a_lane = smem_u32(g_s) + ((mt * 16 + (lane & 15)) * kHPitch + (lane >> 4) * 8) * 2;
    for (int nt = warp >> 2; nt < 3; nt += 2) {
      const uint32_t b_lane = smem_u32(sm + kTW2) + ((nt * 8 + (lane & 7)) * kHPitch + (lane >> 3) * 8) * 2;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kk = 0; kk < 4; kk += 2) {
        uint32_t a0[4], a1[4], bb[4];
        ldsm_x4(a0, a_lane + kk * 32);
        ldsm_x4(a1, a_lane + (kk + 1) * 32);
        ldsm_x4(bb, b_lane + kk * 32);
        const uint32_t b0[2] = {bb[0], bb[1]}, b1[2] = {bb[2], bb[3]};
        mma_bf16(acc, a0, b0);
        mma_bf16(acc, a1, b1);
      }
      const int r0 = mt * 16 + g, j0 = nt * 8 + 2 * t;
      if (j0 < kLabels) {
        logit_s[r0 * kLabels + j0] = acc[0] + fb2[j0];
        logit_s[(r0 + 8) * kLabels + j0] = acc[2] + fb2[j0];
      }
      if (j0 + 1 < kLabels) {
        logit_s[r0 * kLabels + j0 + 1] = acc[1] + fb2[j0 + 1];
        logit_s[(r0 + 8) * kLabels + j0 + 1] = acc[3] + fb2[j0 + 1];
      }
    }
  }
  epi_sync();
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
}

template <typename InT>
__global__ void __launch_bounds__(kBlockT, 1) cnn_infer_tc_kernel(const InferArgs a, int* __restrict__ err,
                                                                   long long wait_limit) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar1;        // conv1 of a pair done
  __shared__ __align__(8) uint64_t bar2, bar3;  // conv2 / conv3 of a pair done
  __shared__ __align__(8) uint64_t e_full[2], e_empty[2];   // expanded-map slots staged / read
  __shared__ __align__(8) uint64_t c1_done, c2_done, c3_done;   // epilogues done (accumulators free, maps written)
  __shared__ __align__(8) uint64_t bar_fin;     // every MMA of the CTA done
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  volatile int* abort = &abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid < kThreadsT) {
    const float* cbs = reinterpret_cast<const float*>(a.packed + kPkCB);
    for (int i = tid; i < 80; i += kThreadsT) reinterpret_cast<float*>(sm + kTCB)[i] = cbs[i];
    const float* hs = reinterpret_cast<const float*>(a.packed + kPkHead);
    float* hd = reinterpret_cast<float*>(sm + kTHead);
    constexpr int nq = kHidden + kHidden * kSlots;
    for (int i = tid; i < nq; i += kThreadsT) hd[i] = hs[i];
    for (int i = tid; i < kLabels * kHidden; i += kThreadsT) hd[nq + (i / kHidden) * kF2Pitch + i % kHidden] = hs[nq + i];
    for (int i = tid; i < kLabels; i += kThreadsT) hd[nq + kLabels * kF2Pitch + i] = hs[nq + kLabels * kHidden + i];
    for (int i = tid; i < 24 * kHPitch; i += kThreadsT) {
      const int j = i / kHPitch, h = i % kHPitch;
      reinterpret_cast<uint16_t*>(sm + kTW2)[i] =
          (j < kLabels && h < kHidden) ? static_cast<uint16_t>(bf16_bits(hs[nq + j * kHidden + h])) : static_cast<uint16_t>(0);
    }
    pack_b_operands(a.packed, sm, tid);
    // zero the activation maps (borders stay zero; interiors are rewritten)
    for (int i = tid; i < (kTFeat - kTAct1) / 16; i += kThreadsT)
      reinterpret_cast<uint4*>(sm + kTAct1)[i] = make_uint4(0, 0, 0, 0);
  }
  if (warp == 0) tmem_alloc(&tmem_base, kTmemColsT);
  if (tid == 0) {
    mbar_init(&bar1, 1);
    mbar_init(&bar2, 1);
    mbar_init(&bar3, 1);
    for (int j = 0; j < 2; ++j) {
      mbar_init(&e_full[j], kProducerWarps);
      mbar_init(&e_empty[j], 1);
    }
    mbar_init(&c1_done, kWarpsT);
    mbar_init(&c2_done, kWarpsT);
    mbar_init(&c3_done, kWarpsT);
    mbar_init(&bar_fin, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  fence_proxy_async_smem();                   // B operands and zeroed maps are read by the tensor cores
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const long long n_groups = (a.n_regions + kGroupT - 1) / kGroupT;
  const long long pairs = (n_groups - blockIdx.x + gridDim.x - 1) / gridDim.x * kPairsT;

  if (warp >= kProducerWarp0) {
    // staging: expanded maps of pair k into slot k % 2, once conv1 of pair k - 2 has read it;
    // warp p does half p % 2 of region p / 2
    const int rs = warp - kProducerWarp0;
    int px0[kStageRows], px1[kStageRows];
    load_half_region<InT>(a, pair_region(a, 0, rs), 0, lane, px0);
    load_half_region<InT>(a, pair_region(a, 0, rs), 1, lane, px1);
    for (long long k = 0; k < pairs; ++k) {
      const int slot = static_cast<int>(k & 1);
      if (k >= 2 && !wait_or_abort(&e_empty[slot], static_cast<uint32_t>(((k - 2) >> 1) & 1), wait_limit, abort)) break;
      store_half_expanded(px0, 0, sm + kTE + (2 * slot + rs) * kEBytes, lane);
      store_half_expanded(px1, 1, sm + kTE + (2 * slot + rs) * kEBytes, lane);
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&e_full[slot]);
      if (k + 1 < pairs) {
        load_half_region<InT>(a, pair_region(a, k + 1, rs), 0, lane, px0);
        load_half_region<InT>(a, pair_region(a, k + 1, rs), 1, lane, px1);
      }
    }
  } else if (warp == kIssuerWarp) {
    // MMA issue: iteration k issues conv1 of pair k, conv2 of pair k - 1, conv3 of pair k - 2
    const uint32_t e_s = smem_u32(sm + kTE), act1_s = smem_u32(sm + kTAct1), act2_s = smem_u32(sm + kTAct2);
    const uint32_t b1_s = smem_u32(sm + kTB1), b2_s = smem_u32(sm + kTB2), b3_s = smem_u32(sm + kTB3);
    constexpr uint32_t idesc64 = idesc_bf16_f32(128, 64), idesc128 = idesc_bf16_f32(128, 128);
    constexpr uint32_t idesc32 = idesc_bf16_f32(128, 32);
    for (long long k = 0; k < pairs + 2; ++k) {
      if (k < pairs) {
        const int slot = static_cast<int>(k & 1);
        if (!wait_or_abort(&e_full[slot], static_cast<uint32_t>((k >> 1) & 1), wait_limit, abort)) break;
        if (k >= 1 && !wait_or_abort(&c1_done, static_cast<uint32_t>((k - 1) & 1), wait_limit, abort)) break;
        tc_fence_after();
        if (lane == 0) {
          // conv1 tile q = (region s, window rows 8 t ..): one MMA of K = 16, N = 64
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            umma_bf16(tmem + kC1Col + 64 * q,
                      umma_desc(e_s + (2 * slot + (q >> 1)) * kEBytes + (q & 1) * 8 * kERow, kERow, 128),
                      umma_desc(b1_s, 128, 256), idesc64, 0u);
            if (q == 3) umma_commit(&bar1);
          }
          umma_commit(&e_empty[slot]);
        }
        __syncwarp();
      } else if (k == pairs) {
        if (!wait_or_abort(&c1_done, static_cast<uint32_t>((k - 1) & 1), wait_limit, abort)) break;
        tc_fence_after();
      }
      if (k >= 1 && k <= pairs) {
        if (k >= 2 && !wait_or_abort(&c2_done, static_cast<uint32_t>((k - 2) & 1), wait_limit, abort)) break;
        tc_fence_after();
        if (lane == 0) {
          // conv2 of pair k - 1: receptive-field offset (ry, rx) of the windows, K = 16 over 2 planes,
          // N = 128 (window pixel x channel; zero weights where the offset is not a tap of that pixel)
          const uint32_t m1 = act1_s + static_cast<uint32_t>((k - 1) & 1) * kAct1T;
#pragma unroll
          for (int off = 0; off < 16; ++off) {
            const int ry = off >> 2, rx = off & 3;
            const uint32_t ab = m1 + (ry & 1) * kRPar + (ry >> 1) * kRP + (rx & 1) * kCPar + (rx >> 1) * 16;
            umma_bf16(tmem + kC2Col, umma_desc(ab, kA1Plane, kRS), umma_desc(b2_s + off * 4096, 128, 256), idesc128,
                      off > 0 ? 1u : 0u);
          }
          umma_commit(&bar2);
        }
        __syncwarp();
      } else if (k == pairs + 1) {
        if (!wait_or_abort(&c2_done, static_cast<uint32_t>((k - 2) & 1), wait_limit, abort)) break;
        tc_fence_after();
      }
      if (k >= 2) {
        if (k >= 3 && !wait_or_abort(&c3_done, static_cast<uint32_t>((k - 3) & 1), wait_limit, abort)) break;
        tc_fence_after();
        if (lane == 0) {
          // conv3 of pair k - 2: 9 taps x 2 channel halves of K = 16, N = 32
          const uint32_t m2 = act2_s + static_cast<uint32_t>(k & 1) * kAct2T;
#pragma unroll
          for (int j = 0; j < 18; ++j) {
            const int tap = j >> 1, h = j & 1;
            umma_bf16(tmem + kC3Col, umma_desc(m2 + ((tap / 3) * 20 + tap % 3) * 16 + 2 * h * kA3Plane, kA3Plane, 160),
                      umma_desc(b3_s + j * 1024, 128, 256), idesc32, j > 0 ? 1u : 0u);
          }
          umma_commit(&bar3);
        }
        __syncwarp();
      }
    }
    // every MMA this thread issued has finished before the tensor memory is freed
    if (lane == 0) umma_commit(&bar_fin);
    __syncwarp();
    if (!mbar_wait_bounded(&bar_fin, 0u, wait_limit)) *abort = 1;
  } else {
    // epilogue warps
    const float* cb = reinterpret_cast<const float*>(sm + kTCB);
    const uint32_t wl = static_cast<uint32_t>((warp & 3) * 32) << 16;   // the warp's tensor-memory lanes
    bool ok = true;
    for (long long k = 0; k < pairs + 2; ++k) {
      if (k < pairs) {
        unsigned char* m1 = sm + kTAct1 + (k & 1) * kAct1T;
        ok &= wait_or_abort(&bar1, static_cast<uint32_t>(k & 1), wait_limit, abort);
        tc_fence_after();
        conv1_epilogue(tmem + wl + kC1Col, m1, cb, warp, lane);
        fence_proxy_async_smem();             // the conv2 input map is read by the tensor cores
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&c1_done);
      }
      if (k >= 1 && k <= pairs) {
        ok &= wait_or_abort(&bar2, static_cast<uint32_t>((k - 1) & 1), wait_limit, abort);
        tc_fence_after();
        conv2_epilogue(tmem + wl + kC2Col, sm + kTAct2 + ((k - 1) & 1) * kAct2T, cb, warp, lane);
        fence_proxy_async_smem();             // the stacked conv3 map is read by the tensor cores
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&c2_done);
      }
      if (k >= 2) {
        const int pr = static_cast<int>((k - 2) % kPairsT);
        ok &= wait_or_abort(&bar3, static_cast<uint32_t>((k - 2) & 1), wait_limit, abort);
        tc_fence_after();
        conv3_epilogue(tmem + wl + kC3Col, sm + kTFeat + 2 * pr * kFeatPitch * 2, cb, warp, lane);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&c3_done);
        if (pr == kPairsT - 1) {              // the group of pair k - 2 is complete
          if (!epi_sync_and(ok && *abort == 0)) break;
          const long long n = (k - 2) / kPairsT;
          group_head(a, (static_cast<long long>(blockIdx.x) + n * gridDim.x) * kGroupT, sm, tid);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && abort_flag) atomicOr(err, 2);
  if (warp == 0) tmem_dealloc(tmem, kTmemColsT);
}

template <typename InT>
int launch_infer_tc_t(const InferArgs& a, int num_sms, int* err, void* stream) {
  auto kern = cnn_infer_tc_kernel<InT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemT);
  if (e != cudaSuccess) return static_cast<int>(e);
  const long long groups = (a.n_regions + kGroupT - 1) / kGroupT;
  const int grid = static_cast<int>(groups < num_sms ? groups : num_sms);
  if (grid <= 0) return 0;
  long long limit = kDefaultWaitLimit;
  (void)fault_mode(&limit);
  kern<<<grid, kBlockT, kSmemT, static_cast<cudaStream_t>(stream)>>>(a, err, limit);
  return static_cast<int>(cudaGetLastError());
}
