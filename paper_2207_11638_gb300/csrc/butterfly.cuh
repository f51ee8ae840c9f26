// Register butterflies for the Chen-factorization DCT approximations.
//
// Every function here applies one matrix of the paper's fast algorithms to a
// small array held in registers, in place.  Indices are compile-time
// constants after unrolling, so each function becomes straight-line integer
// adds (and, for the exact DCT, float multiply-adds); multiplications by the
// integer parameters 0 and 1 fold away, and x2 folds into a shift-add.
//
// Notation follows arXiv 2207.11638:
//   T_C(alpha, beta, gamma) = P_8 M_1 M_2 M_3 M_4 B_8                  (Sec. 3)
//   T~_8 = T_C(sign(...)), T^_8 = T_C(round(...))                      (Eqs. 4-5)
//   T_8^{-1} = 1/2 B_8^T M_4^{-1} M_3^{-1} M_2^{-1} M_1^T P_8^T        (Eqs. 6-7)
//   T_N = M^per_N diag(T_{N/2}, T_{N/2}) M^add_N,  N = 16, 32          (Eq. app_N)
// The integer inverse is carried as W_N = 2 U_N = 2 N T_N^{-1}:
//   W_8 = B_8 (2M_4^{-1}) (2M_3^{-1}) (2M_2^{-1}) M_1^T P_8^T          (integer stages)
//   W_N = M^add_N diag(W_{N/2}, W_{N/2}) (M^per_N)^T
// which needs no halving anywhere; the final power-of-two scale absorbs it.
#pragma once

#define CDCT_DEV __host__ __device__ __forceinline__

namespace cdct {

// ---------------------------------------------------------------------------
// Parameter sets (alpha, beta_0..3, gamma_0..1) of Sec. 3.
// ---------------------------------------------------------------------------
struct ParamsTilde {  // sign() of the Chen constants: all ones
  typedef int T;
  static constexpr int a = 1, b0 = 1, b1 = 1, b2 = 1, b3 = 1, g0 = 1, g1 = 1;
};
struct ParamsHat {    // round() of the Chen constants: beta_3 = gamma_1 = 0
  typedef int T;
  static constexpr int a = 1, b0 = 1, b1 = 1, b2 = 1, b3 = 0, g0 = 1, g1 = 0;
};
struct ParamsExact {  // cos(pi/4), cos((2n+1) pi/16), cos((2n+1) pi/8)
  typedef float T;
  static constexpr float a = 0.70710678118654752f;
  static constexpr float b0 = 0.98078528040323044f, b1 = 0.83146961230254524f;
  static constexpr float b2 = 0.55557023301960222f, b3 = 0.19509032201612826f;
  static constexpr float g0 = 0.92387953251128674f, g1 = 0.38268343236508977f;
};

// ---------------------------------------------------------------------------
// Forward stages of T_C (Eq. 3 factor matrices), x <- M x.
// ---------------------------------------------------------------------------
template <typename T>
CDCT_DEV void st_B8(T (&x)[8]) {  // B_8 = [[I_4, I-bar_4], [I-bar_4, -I_4]] (symmetric)
  T y[8];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    y[i] = x[i] + x[7 - i];
    y[4 + i] = x[3 - i] - x[4 + i];
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = y[i];
}

template <class P, typename T>
CDCT_DEV void st_M4(T (&x)[8]) {  // M_4 = diag(B_4, A_3(alpha))
  T y0 = x[0] + x[3], y1 = x[1] + x[2], y2 = x[1] - x[2], y3 = x[0] - x[3];
  T y4 = x[7], y5 = P::a * (x[5] + x[6]), y6 = P::a * (x[6] - x[5]), y7 = x[4];
  x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3; x[4] = y4; x[5] = y5; x[6] = y6; x[7] = y7;
}

template <class P, typename T>
CDCT_DEV void st_M4t(T (&x)[8]) {  // M_4^T = diag(B_4, A_3^T)
  T y0 = x[0] + x[3], y1 = x[1] + x[2], y2 = x[1] - x[2], y3 = x[0] - x[3];
  T y4 = x[7], y5 = P::a * (x[5] - x[6]), y6 = P::a * (x[5] + x[6]), y7 = x[4];
  x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3; x[4] = y4; x[5] = y5; x[6] = y6; x[7] = y7;
}

template <class P, typename T>
CDCT_DEV void st_M3(T (&x)[8]) {  // M_3 = diag(C-tilde(alpha, gamma), A_2) (symmetric)
  T y0 = P::a * (x[0] + x[1]), y1 = P::a * (x[0] - x[1]);
  T y2 = P::g1 * x[3] - P::g0 * x[2], y3 = P::g1 * x[2] + P::g0 * x[3];
  T y4 = x[4] + x[5], y5 = x[4] - x[5], y6 = x[7] - x[6], y7 = x[6] + x[7];
  x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3; x[4] = y4; x[5] = y5; x[6] = y6; x[7] = y7;
}

template <class P, typename T>
CDCT_DEV void st_M2(T (&x)[8]) {  // M_2 = diag(P_4, A_1(beta)) (A_1 symmetric)
  T y0 = x[0], y1 = x[3], y2 = x[1], y3 = x[2];
  T y4 = P::b0 * x[4] + P::b3 * x[7], y5 = P::b2 * x[5] + P::b1 * x[6];
  T y6 = P::b1 * x[5] - P::b2 * x[6], y7 = P::b3 * x[4] - P::b0 * x[7];
  x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3; x[4] = y4; x[5] = y5; x[6] = y6; x[7] = y7;
}

template <class P, typename T>
CDCT_DEV void st_M2t(T (&x)[8]) {  // M_2^T = diag(P_4^T, A_1)
  T y0 = x[0], y3 = x[1], y1 = x[2], y2 = x[3];
  T y4 = P::b0 * x[4] + P::b3 * x[7], y5 = P::b2 * x[5] + P::b1 * x[6];
  T y6 = P::b1 * x[5] - P::b2 * x[6], y7 = P::b3 * x[4] - P::b0 * x[7];
  x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3; x[4] = y4; x[5] = y5; x[6] = y6; x[7] = y7;
}

template <typename T>
CDCT_DEV void st_M1(T (&x)[8]) {  // M_1 = diag(I_4, I-bar_4 Q): swaps entries 4 and 7 (= M_1^T)
  T t = x[4]; x[4] = x[7]; x[7] = t;
}

template <typename T>
CDCT_DEV void st_P8(T (&x)[8]) {  // P_8: rows pick 0,7,1,6,2,5,3,4
  T y[8] = {x[0], x[7], x[1], x[6], x[2], x[5], x[3], x[4]};
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = y[i];
}

template <typename T>
CDCT_DEV void st_P8t(T (&x)[8]) {  // P_8^T
  T y[8];
  y[0] = x[0]; y[7] = x[1]; y[1] = x[2]; y[6] = x[3];
  y[2] = x[4]; y[5] = x[5]; y[3] = x[6]; y[4] = x[7];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = y[i];
}

// ---------------------------------------------------------------------------
// Doubled inverse stages 2 M_i^{-1} (Eqs. 6-7), integer parameters only.
// With A_1^2 = diag(b0^2+b3^2, b1^2+b2^2, b1^2+b2^2, b0^2+b3^2),
// 2 A_1^{-1} = A_1 diag(k03, k12, k12, k03) with k = 2 / (sum of squares);
// 2 C-tilde^{-1} uses kg = 2 / (g0^2 + g1^2) on its gamma block.
// ---------------------------------------------------------------------------
template <class P>
struct InvK {
  static_assert(P::a == 1, "integer inverse stages assume alpha = 1");
  static constexpr int k03 = 2 / (P::b0 * P::b0 + P::b3 * P::b3);
  static constexpr int k12 = 2 / (P::b1 * P::b1 + P::b2 * P::b2);
  static constexpr int kg = 2 / (P::g0 * P::g0 + P::g1 * P::g1);
};

template <class P, typename V>
CDCT_DEV void st_2M2inv(V (&x)[8]) {  // 2 M_2^{-1} = diag(2 P_4^T, 2 A_1^{-1})
  typedef InvK<P> K;
  V y0 = 2 * x[0], y1 = 2 * x[2], y2 = 2 * x[3], y3 = 2 * x[1];
  V s4 = K::k03 * x[4], s5 = K::k12 * x[5], s6 = K::k12 * x[6], s7 = K::k03 * x[7];
  V y4 = P::b0 * s4 + P::b3 * s7, y5 = P::b2 * s5 + P::b1 * s6;
  V y6 = P::b1 * s5 - P::b2 * s6, y7 = P::b3 * s4 - P::b0 * s7;
  x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3; x[4] = y4; x[5] = y5; x[6] = y6; x[7] = y7;
}

template <class P, typename V>
CDCT_DEV void st_2M2inv_t(V (&x)[8]) {  // (2 M_2^{-1})^T = diag(2 P_4, diag(k) A_1)
  typedef InvK<P> K;
  V y0 = 2 * x[0], y1 = 2 * x[3], y2 = 2 * x[1], y3 = 2 * x[2];
  V y4 = K::k03 * (P::b0 * x[4] + P::b3 * x[7]);
  V y5 = K::k12 * (P::b2 * x[5] + P::b1 * x[6]);
  V y6 = K::k12 * (P::b1 * x[5] - P::b2 * x[6]);
  V y7 = K::k03 * (P::b3 * x[4] - P::b0 * x[7]);
  x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3; x[4] = y4; x[5] = y5; x[6] = y6; x[7] = y7;
}

template <class P, typename V>
CDCT_DEV void st_2M3inv(V (&x)[8]) {  // 2 M_3^{-1} = diag(2 C-tilde^{-1}, A_2) (symmetric)
  typedef InvK<P> K;
  V y0 = x[0] + x[1], y1 = x[0] - x[1];
  V y2 = K::kg * (P::g1 * x[3] - P::g0 * x[2]), y3 = K::kg * (P::g1 * x[2] + P::g0 * x[3]);
  V y4 = x[4] + x[5], y5 = x[4] - x[5], y6 = x[7] - x[6], y7 = x[6] + x[7];
  x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3; x[4] = y4; x[5] = y5; x[6] = y6; x[7] = y7;
}

template <class P, typename V>
CDCT_DEV void st_2M4inv(V (&x)[8]) {  // 2 M_4^{-1} = diag(B_4, 2 A_3^{-1})
  V y0 = x[0] + x[3], y1 = x[1] + x[2], y2 = x[1] - x[2], y3 = x[0] - x[3];
  V y4 = 2 * x[7], y5 = x[5] - x[6], y6 = x[5] + x[6], y7 = 2 * x[4];
  x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3; x[4] = y4; x[5] = y5; x[6] = y6; x[7] = y7;
}

template <class P, typename V>
CDCT_DEV void st_2M4inv_t(V (&x)[8]) {  // (2 M_4^{-1})^T = diag(B_4, 2 A_3^{-T})
  V y0 = x[0] + x[3], y1 = x[1] + x[2], y2 = x[1] - x[2], y3 = x[0] - x[3];
  V y4 = 2 * x[7], y5 = x[5] + x[6], y6 = x[6] - x[5], y7 = 2 * x[4];
  x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3; x[4] = y4; x[5] = y5; x[6] = y6; x[7] = y7;
}

// ---------------------------------------------------------------------------
// 8-point operators.
// ---------------------------------------------------------------------------
template <class P, typename T>
CDCT_DEV void T8_apply(T (&x)[8]) {  // x <- T_C x = P_8 M_1 M_2 M_3 M_4 B_8 x
  st_B8(x); st_M4<P>(x); st_M3<P>(x); st_M2<P>(x); st_M1(x); st_P8(x);
}

template <class P, typename T>
CDCT_DEV void T8t_apply(T (&x)[8]) {  // x <- T_C^T x = B_8 M_4^T M_3 M_2^T M_1 P_8^T x
  st_P8t(x); st_M1(x); st_M2t<P>(x); st_M3<P>(x); st_M4t<P>(x); st_B8(x);
}

template <class P, typename V>
CDCT_DEV void W8_apply(V (&x)[8]) {  // x <- 2 U_8 x = B_8 (2M_4^-1)(2M_3^-1)(2M_2^-1) M_1 P_8^T x
  st_P8t(x); st_M1(x); st_2M2inv<P, V>(x); st_2M3inv<P, V>(x); st_2M4inv<P, V>(x); st_B8(x);
}

template <class P, typename V>
CDCT_DEV void W8t_apply(V (&x)[8]) {  // x <- 2 U_8^T x = P_8 M_1 (2M_2^-1)^T (2M_3^-1) (2M_4^-1)^T B_8 x
  st_B8(x); st_2M4inv_t<P, V>(x); st_2M3inv<P, V>(x); st_2M2inv_t<P, V>(x); st_M1(x); st_P8(x);
}

// ---------------------------------------------------------------------------
// JAM recursion (Sec. 6): M^add_N = [[I, I-bar], [I-bar, -I]] (symmetric),
// M^per_N interleaves the halves (row 2k <- upper k, row 2k+1 <- lower k).
// ---------------------------------------------------------------------------
template <int N, typename V>
CDCT_DEV void madd(V (&x)[N], V (&lo)[N / 2], V (&hi)[N / 2]) {  // (lo; hi) = M^add x
#pragma unroll
  for (int k = 0; k < N / 2; ++k) {
    lo[k] = x[k] + x[N - 1 - k];
    hi[k] = x[N / 2 - 1 - k] - x[N / 2 + k];
  }
}

template <int N, typename V>
CDCT_DEV void madd_join(V (&lo)[N / 2], V (&hi)[N / 2], V (&x)[N]) {  // x = M^add (lo; hi)
#pragma unroll
  for (int k = 0; k < N / 2; ++k) {
    x[k] = lo[k] + hi[N / 2 - 1 - k];
    x[N / 2 + k] = lo[N / 2 - 1 - k] - hi[k];
  }
}

template <int N, typename V>
CDCT_DEV void interleave(V (&lo)[N / 2], V (&hi)[N / 2], V (&x)[N]) {  // x = M^per (lo; hi)
#pragma unroll
  for (int k = 0; k < N / 2; ++k) { x[2 * k] = lo[k]; x[2 * k + 1] = hi[k]; }
}

template <int N, typename V>
CDCT_DEV void deinterleave(V (&x)[N], V (&lo)[N / 2], V (&hi)[N / 2]) {  // (lo; hi) = M^per^T x
#pragma unroll
  for (int k = 0; k < N / 2; ++k) { lo[k] = x[2 * k]; hi[k] = x[2 * k + 1]; }
}

template <int N, class P>
struct Jam {
  // x <- T_N x = M^per diag(T_{N/2}, T_{N/2}) M^add x
  template <typename V>
  static CDCT_DEV void T(V (&x)[N]) {
    V lo[N / 2], hi[N / 2];
    madd<N>(x, lo, hi);
    Jam<N / 2, P>::T(lo);
    Jam<N / 2, P>::T(hi);
    interleave<N>(lo, hi, x);
  }
  // x <- T_N^T x = M^add diag(T_{N/2}^T, T_{N/2}^T) M^per^T x
  template <typename V>
  static CDCT_DEV void Tt(V (&x)[N]) {
    V lo[N / 2], hi[N / 2];
    deinterleave<N>(x, lo, hi);
    Jam<N / 2, P>::Tt(lo);
    Jam<N / 2, P>::Tt(hi);
    madd_join<N>(lo, hi, x);
  }
  // x <- W_N x = M^add diag(W_{N/2}, W_{N/2}) M^per^T x   (W_N = 2 N T_N^{-1})
  template <typename V>
  static CDCT_DEV void W(V (&x)[N]) {
    V lo[N / 2], hi[N / 2];
    deinterleave<N>(x, lo, hi);
    Jam<N / 2, P>::W(lo);
    Jam<N / 2, P>::W(hi);
    madd_join<N>(lo, hi, x);
  }
  // x <- W_N^T x = M^per diag(W_{N/2}^T, W_{N/2}^T) M^add x
  template <typename V>
  static CDCT_DEV void Wt(V (&x)[N]) {
    V lo[N / 2], hi[N / 2];
    madd<N>(x, lo, hi);
    Jam<N / 2, P>::Wt(lo);
    Jam<N / 2, P>::Wt(hi);
    interleave<N>(lo, hi, x);
  }
};

template <class P>
struct Jam<8, P> {
  template <typename V>
  static CDCT_DEV void T(V (&x)[8]) { T8_apply<P>(x); }
  template <typename V>
  static CDCT_DEV void Tt(V (&x)[8]) { T8t_apply<P>(x); }
  template <typename V>
  static CDCT_DEV void W(V (&x)[8]) { W8_apply<P>(x); }
  template <typename V>
  static CDCT_DEV void Wt(V (&x)[8]) { W8t_apply<P>(x); }
};

}  // namespace cdct
