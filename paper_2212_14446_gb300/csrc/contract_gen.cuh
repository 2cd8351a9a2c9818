// Generated by gen_contract.py -- do not edit.
// Angular monomials (Eq. 23b, Table 3), three-body contraction (Eq. 26a, Table 4),
// four-body contraction (Eq. 27a, Eq. 30a) and their adjoints, unrolled per PA.
#pragma once
template <int PA> struct Mono;
template <int PA> struct Four;
template <> struct Mono<0> {
  static constexpr int NA = 1;
  template <typename T>
  static __device__ __forceinline__ void eval(T ux, T uy, T uz, T* A) {
    A[0] = T(1);
  }
  static constexpr int NA2 = 1;
  static __device__ __forceinline__ void eval2(float ux, float uy, float uz, float2* A2) {
    A2[0].x = 1.0f;
    A2[0].y = 0.0f;
  }
  template <typename T>
  static __device__ __forceinline__ void eval_d(T ux, T uy, T uz, T wx, T wy, T wz, T* A, T* dA) {
    A[0] = T(1);
    dA[0] = T(0);
  }
  template <typename T>
  static __device__ __forceinline__ void grad(const T* e, const T* A, T& gx, T& gy, T& gz) {
    T g0 = T(0), g1 = T(0), g2 = T(0);
    gx = g0; gy = g1; gz = g2;
  }
  template <typename T>
  static __device__ __forceinline__ void dot_grad_deg(const T* e, const T* A, T* s, T* gx, T* gy, T* gz) {
    for (int n = 0; n <= 0; ++n) { s[n] = T(0); gx[n] = T(0); gy[n] = T(0); gz[n] = T(0); }
    s[0] = fma(e[0], A[0], s[0]);
  }
  template <typename T>
  static __device__ __forceinline__ void d3(const T* B, T* d) {
    d[0] = B[0] * B[0];
  }
  template <typename T>
  static __device__ __forceinline__ void d3_tangent(const T* B, const T* Bd, T* d) {
    d[0] = T(2) * B[0] * Bd[0];
  }
  template <typename T>
  static __device__ __forceinline__ void d3_adjoint(const T* B, const T* h, T* a) {
    a[0] = fma(T(2) * h[0], B[0], a[0]);
  }
};
template <> struct Four<0> {
  static constexpr int KA = 1;
  static __device__ __forceinline__ int p_n00(int n) {
    switch (n) {
      case 0: return 0;
      default: return -1;
    }
  }
  template <typename T>
  static __device__ __forceinline__ void desc(const T* B, const T* d3, T* D) {
    D[0] = B[0] * d3[0];
  }
  template <typename T>
  static __device__ __forceinline__ void adjoint(const T* B, const T* w, T* a) {
  }
  template <typename T>
  static __device__ __forceinline__ void tangent(const T* B, const T* Bd, const T* d3, const T* d3d, T* Dd) {
    Dd[0] = fma(Bd[0], d3[0], B[0] * d3d[0]);
  }
  static constexpr int NTERMS = 0;
};
template <> struct Mono<1> {
  static constexpr int NA = 4;
  template <typename T>
  static __device__ __forceinline__ void eval(T ux, T uy, T uz, T* A) {
    A[0] = T(1);
    A[1] = ux;
    A[2] = uy;
    A[3] = uz;
  }
  static constexpr int NA2 = 2;
  static __device__ __forceinline__ void eval2(float ux, float uy, float uz, float2* A2) {
    A2[0].x = 1.0f;
    A2[0].y = ux;
    A2[1].x = uy;
    A2[1].y = uz;
  }
  template <typename T>
  static __device__ __forceinline__ void eval_d(T ux, T uy, T uz, T wx, T wy, T wz, T* A, T* dA) {
    A[0] = T(1);
    dA[0] = T(0);
    A[1] = ux;
    dA[1] = wx;
    A[2] = uy;
    dA[2] = wy;
    A[3] = uz;
    dA[3] = wz;
  }
  template <typename T>
  static __device__ __forceinline__ void grad(const T* e, const T* A, T& gx, T& gy, T& gz) {
    T g0 = T(0), g1 = T(0), g2 = T(0);
    g0 = fma(e[1], A[0], g0);
    g1 = fma(e[2], A[0], g1);
    g2 = fma(e[3], A[0], g2);
    gx = g0; gy = g1; gz = g2;
  }
  template <typename T>
  static __device__ __forceinline__ void dot_grad_deg(const T* e, const T* A, T* s, T* gx, T* gy, T* gz) {
    for (int n = 0; n <= 1; ++n) { s[n] = T(0); gx[n] = T(0); gy[n] = T(0); gz[n] = T(0); }
    s[0] = fma(e[0], A[0], s[0]);
    s[1] = fma(e[1], A[1], s[1]);
    gx[1] = fma(e[1], A[0], gx[1]);
    s[1] = fma(e[2], A[2], s[1]);
    gy[1] = fma(e[2], A[0], gy[1]);
    s[1] = fma(e[3], A[3], s[1]);
    gz[1] = fma(e[3], A[0], gz[1]);
  }
  template <typename T>
  static __device__ __forceinline__ void d3(const T* B, T* d) {
    d[0] = B[0] * B[0];
    d[1] = B[1] * B[1] + B[2] * B[2] + B[3] * B[3];
  }
  template <typename T>
  static __device__ __forceinline__ void d3_tangent(const T* B, const T* Bd, T* d) {
    d[0] = T(2) * B[0] * Bd[0];
    d[1] = T(2) * B[1] * Bd[1] + T(2) * B[2] * Bd[2] + T(2) * B[3] * Bd[3];
  }
  template <typename T>
  static __device__ __forceinline__ void d3_adjoint(const T* B, const T* h, T* a) {
    a[0] = fma(T(2) * h[0], B[0], a[0]);
    a[1] = fma(T(2) * h[1], B[1], a[1]);
    a[2] = fma(T(2) * h[1], B[2], a[2]);
    a[3] = fma(T(2) * h[1], B[3], a[3]);
  }
};
template <> struct Four<1> {
  static constexpr int KA = 2;
  static __device__ __forceinline__ int p_n00(int n) {
    switch (n) {
      case 0: return 0;
      case 1: return 1;
      default: return -1;
    }
  }
  template <typename T>
  static __device__ __forceinline__ void desc(const T* B, const T* d3, T* D) {
    D[0] = B[0] * d3[0];
    D[1] = B[0] * d3[1];
  }
  template <typename T>
  static __device__ __forceinline__ void adjoint(const T* B, const T* w, T* a) {
  }
  template <typename T>
  static __device__ __forceinline__ void tangent(const T* B, const T* Bd, const T* d3, const T* d3d, T* Dd) {
    Dd[0] = fma(Bd[0], d3[0], B[0] * d3d[0]);
    Dd[1] = fma(Bd[0], d3[1], B[0] * d3d[1]);
  }
  static constexpr int NTERMS = 0;
};
template <> struct Mono<2> {
  static constexpr int NA = 10;
  template <typename T>
  static __device__ __forceinline__ void eval(T ux, T uy, T uz, T* A) {
    A[0] = T(1);
    A[1] = ux;
    A[2] = uy;
    A[3] = uz;
    A[4] = A[1] * ux;
    A[5] = A[2] * uy;
    A[6] = A[3] * uz;
    A[7] = A[2] * ux;
    A[8] = A[3] * ux;
    A[9] = A[3] * uy;
  }
  static constexpr int NA2 = 5;
  static __device__ __forceinline__ void eval2(float ux, float uy, float uz, float2* A2) {
    A2[0].x = 1.0f;
    A2[0].y = ux;
    A2[1].x = uy;
    A2[1].y = uz;
    A2[2].x = A2[0].y * ux;
    A2[2].y = A2[1].x * uy;
    A2[3].x = A2[1].y * uz;
    A2[3].y = A2[1].x * ux;
    A2[4].x = A2[1].y * ux;
    A2[4].y = A2[1].y * uy;
  }
  template <typename T>
  static __device__ __forceinline__ void eval_d(T ux, T uy, T uz, T wx, T wy, T wz, T* A, T* dA) {
    A[0] = T(1);
    dA[0] = T(0);
    A[1] = ux;
    dA[1] = wx;
    A[2] = uy;
    dA[2] = wy;
    A[3] = uz;
    dA[3] = wz;
    A[4] = A[1] * ux;
    dA[4] = fma(dA[1], ux, A[1] * wx);
    A[5] = A[2] * uy;
    dA[5] = fma(dA[2], uy, A[2] * wy);
    A[6] = A[3] * uz;
    dA[6] = fma(dA[3], uz, A[3] * wz);
    A[7] = A[2] * ux;
    dA[7] = fma(dA[2], ux, A[2] * wx);
    A[8] = A[3] * ux;
    dA[8] = fma(dA[3], ux, A[3] * wx);
    A[9] = A[3] * uy;
    dA[9] = fma(dA[3], uy, A[3] * wy);
  }
  template <typename T>
  static __device__ __forceinline__ void grad(const T* e, const T* A, T& gx, T& gy, T& gz) {
    T g0 = T(0), g1 = T(0), g2 = T(0);
    g0 = fma(e[1], A[0], g0);
    g1 = fma(e[2], A[0], g1);
    g2 = fma(e[3], A[0], g2);
    g0 = fma(T(2) * e[4], A[1], g0);
    g1 = fma(T(2) * e[5], A[2], g1);
    g2 = fma(T(2) * e[6], A[3], g2);
    g0 = fma(e[7], A[2], g0);
    g1 = fma(e[7], A[1], g1);
    g0 = fma(e[8], A[3], g0);
    g2 = fma(e[8], A[1], g2);
    g1 = fma(e[9], A[3], g1);
    g2 = fma(e[9], A[2], g2);
    gx = g0; gy = g1; gz = g2;
  }
  template <typename T>
  static __device__ __forceinline__ void dot_grad_deg(const T* e, const T* A, T* s, T* gx, T* gy, T* gz) {
    for (int n = 0; n <= 2; ++n) { s[n] = T(0); gx[n] = T(0); gy[n] = T(0); gz[n] = T(0); }
    s[0] = fma(e[0], A[0], s[0]);
    s[1] = fma(e[1], A[1], s[1]);
    gx[1] = fma(e[1], A[0], gx[1]);
    s[1] = fma(e[2], A[2], s[1]);
    gy[1] = fma(e[2], A[0], gy[1]);
    s[1] = fma(e[3], A[3], s[1]);
    gz[1] = fma(e[3], A[0], gz[1]);
    s[2] = fma(e[4], A[4], s[2]);
    gx[2] = fma(T(2) * e[4], A[1], gx[2]);
    s[2] = fma(e[5], A[5], s[2]);
    gy[2] = fma(T(2) * e[5], A[2], gy[2]);
    s[2] = fma(e[6], A[6], s[2]);
    gz[2] = fma(T(2) * e[6], A[3], gz[2]);
    s[2] = fma(e[7], A[7], s[2]);
    gx[2] = fma(e[7], A[2], gx[2]);
    gy[2] = fma(e[7], A[1], gy[2]);
    s[2] = fma(e[8], A[8], s[2]);
    gx[2] = fma(e[8], A[3], gx[2]);
    gz[2] = fma(e[8], A[1], gz[2]);
    s[2] = fma(e[9], A[9], s[2]);
    gy[2] = fma(e[9], A[3], gy[2]);
    gz[2] = fma(e[9], A[2], gz[2]);
  }
  template <typename T>
  static __device__ __forceinline__ void d3(const T* B, T* d) {
    d[0] = B[0] * B[0];
    d[1] = B[1] * B[1] + B[2] * B[2] + B[3] * B[3];
    d[2] = B[4] * B[4] + B[5] * B[5] + B[6] * B[6] + T(2) * B[7] * B[7] + T(2) * B[8] * B[8] + T(2) * B[9] * B[9];
  }
  template <typename T>
  static __device__ __forceinline__ void d3_tangent(const T* B, const T* Bd, T* d) {
    d[0] = T(2) * B[0] * Bd[0];
    d[1] = T(2) * B[1] * Bd[1] + T(2) * B[2] * Bd[2] + T(2) * B[3] * Bd[3];
    d[2] = T(2) * B[4] * Bd[4] + T(2) * B[5] * Bd[5] + T(2) * B[6] * Bd[6] + T(4) * B[7] * Bd[7] + T(4) * B[8] * Bd[8] + T(4) * B[9] * Bd[9];
  }
  template <typename T>
  static __device__ __forceinline__ void d3_adjoint(const T* B, const T* h, T* a) {
    a[0] = fma(T(2) * h[0], B[0], a[0]);
    a[1] = fma(T(2) * h[1], B[1], a[1]);
    a[2] = fma(T(2) * h[1], B[2], a[2]);
    a[3] = fma(T(2) * h[1], B[3], a[3]);
    a[4] = fma(T(2) * h[2], B[4], a[4]);
    a[5] = fma(T(2) * h[2], B[5], a[5]);
    a[6] = fma(T(2) * h[2], B[6], a[6]);
    a[7] = fma(T(4) * h[2], B[7], a[7]);
    a[8] = fma(T(4) * h[2], B[8], a[8]);
    a[9] = fma(T(4) * h[2], B[9], a[9]);
  }
};
template <> struct Four<2> {
  static constexpr int KA = 4;
  static __device__ __forceinline__ int p_n00(int n) {
    switch (n) {
      case 0: return 0;
      case 1: return 1;
      case 2: return 2;
      default: return -1;
    }
  }
  template <typename T>
  static __device__ __forceinline__ void desc(const T* B, const T* d3, T* D) {
    D[0] = B[0] * d3[0];
    D[1] = B[0] * d3[1];
    D[2] = B[0] * d3[2];
    D[3] = B[1] * B[1] * B[4] + T(2) * B[1] * B[2] * B[7] + T(2) * B[1] * B[3] * B[8] + B[2] * B[2] * B[5] + T(2) * B[2] * B[3] * B[9] + B[3] * B[3] * B[6];
  }
  template <typename T>
  static __device__ __forceinline__ void adjoint(const T* B, const T* w, T* a) {
    {
      const T wp = w[3];
      a[1] = fma(wp, B[1] * B[4], a[1]);
      a[1] = fma(wp, B[1] * B[4], a[1]);
      a[4] = fma(wp, B[1] * B[1], a[4]);
      const T wk1_2_7 = T(2) * wp;
      a[1] = fma(wk1_2_7, B[2] * B[7], a[1]);
      a[2] = fma(wk1_2_7, B[1] * B[7], a[2]);
      a[7] = fma(wk1_2_7, B[1] * B[2], a[7]);
      const T wk1_3_8 = T(2) * wp;
      a[1] = fma(wk1_3_8, B[3] * B[8], a[1]);
      a[3] = fma(wk1_3_8, B[1] * B[8], a[3]);
      a[8] = fma(wk1_3_8, B[1] * B[3], a[8]);
      a[2] = fma(wp, B[2] * B[5], a[2]);
      a[2] = fma(wp, B[2] * B[5], a[2]);
      a[5] = fma(wp, B[2] * B[2], a[5]);
      const T wk2_3_9 = T(2) * wp;
      a[2] = fma(wk2_3_9, B[3] * B[9], a[2]);
      a[3] = fma(wk2_3_9, B[2] * B[9], a[3]);
      a[9] = fma(wk2_3_9, B[2] * B[3], a[9]);
      a[3] = fma(wp, B[3] * B[6], a[3]);
      a[3] = fma(wp, B[3] * B[6], a[3]);
      a[6] = fma(wp, B[3] * B[3], a[6]);
    }
  }
  template <typename T>
  static __device__ __forceinline__ void tangent(const T* B, const T* Bd, const T* d3, const T* d3d, T* Dd) {
    Dd[0] = fma(Bd[0], d3[0], B[0] * d3d[0]);
    Dd[1] = fma(Bd[0], d3[1], B[0] * d3d[1]);
    Dd[2] = fma(Bd[0], d3[2], B[0] * d3d[2]);
    Dd[3] = (Bd[1] * B[1] * B[4] + B[1] * Bd[1] * B[4] + B[1] * B[1] * Bd[4]) + T(2) * (Bd[1] * B[2] * B[7] + B[1] * Bd[2] * B[7] + B[1] * B[2] * Bd[7]) + T(2) * (Bd[1] * B[3] * B[8] + B[1] * Bd[3] * B[8] + B[1] * B[3] * Bd[8]) + (Bd[2] * B[2] * B[5] + B[2] * Bd[2] * B[5] + B[2] * B[2] * Bd[5]) + T(2) * (Bd[2] * B[3] * B[9] + B[2] * Bd[3] * B[9] + B[2] * B[3] * Bd[9]) + (Bd[3] * B[3] * B[6] + B[3] * Bd[3] * B[6] + B[3] * B[3] * Bd[6]);
  }
  static constexpr int NTERMS = 6;
};
template <> struct Mono<3> {
  static constexpr int NA = 20;
  template <typename T>
  static __device__ __forceinline__ void eval(T ux, T uy, T uz, T* A) {
    A[0] = T(1);
    A[1] = ux;
    A[2] = uy;
    A[3] = uz;
    A[4] = A[1] * ux;
    A[5] = A[2] * uy;
    A[6] = A[3] * uz;
    A[7] = A[2] * ux;
    A[8] = A[3] * ux;
    A[9] = A[3] * uy;
    A[10] = A[4] * ux;
    A[11] = A[5] * uy;
    A[12] = A[6] * uz;
    A[13] = A[7] * ux;
    A[14] = A[8] * ux;
    A[15] = A[5] * ux;
    A[16] = A[9] * uy;
    A[17] = A[6] * ux;
    A[18] = A[6] * uy;
    A[19] = A[9] * ux;
  }
  static constexpr int NA2 = 10;
  static __device__ __forceinline__ void eval2(float ux, float uy, float uz, float2* A2) {
    A2[0].x = 1.0f;
    A2[0].y = ux;
    A2[1].x = uy;
    A2[1].y = uz;
    A2[2].x = A2[0].y * ux;
    A2[2].y = A2[1].x * uy;
    A2[3].x = A2[1].y * uz;
    A2[3].y = A2[1].x * ux;
    A2[4].x = A2[1].y * ux;
    A2[4].y = A2[1].y * uy;
    A2[5].x = A2[2].x * ux;
    A2[5].y = A2[2].y * uy;
    A2[6].x = A2[3].x * uz;
    A2[6].y = A2[3].y * ux;
    A2[7].x = A2[4].x * ux;
    A2[7].y = A2[2].y * ux;
    A2[8].x = A2[4].y * uy;
    A2[8].y = A2[3].x * ux;
    A2[9].x = A2[3].x * uy;
    A2[9].y = A2[4].y * ux;
  }
  template <typename T>
  static __device__ __forceinline__ void eval_d(T ux, T uy, T uz, T wx, T wy, T wz, T* A, T* dA) {
    A[0] = T(1);
    dA[0] = T(0);
    A[1] = ux;
    dA[1] = wx;
    A[2] = uy;
    dA[2] = wy;
    A[3] = uz;
    dA[3] = wz;
    A[4] = A[1] * ux;
    dA[4] = fma(dA[1], ux, A[1] * wx);
    A[5] = A[2] * uy;
    dA[5] = fma(dA[2], uy, A[2] * wy);
    A[6] = A[3] * uz;
    dA[6] = fma(dA[3], uz, A[3] * wz);
    A[7] = A[2] * ux;
    dA[7] = fma(dA[2], ux, A[2] * wx);
    A[8] = A[3] * ux;
    dA[8] = fma(dA[3], ux, A[3] * wx);
    A[9] = A[3] * uy;
    dA[9] = fma(dA[3], uy, A[3] * wy);
    A[10] = A[4] * ux;
    dA[10] = fma(dA[4], ux, A[4] * wx);
    A[11] = A[5] * uy;
    dA[11] = fma(dA[5], uy, A[5] * wy);
    A[12] = A[6] * uz;
    dA[12] = fma(dA[6], uz, A[6] * wz);
    A[13] = A[7] * ux;
    dA[13] = fma(dA[7], ux, A[7] * wx);
    A[14] = A[8] * ux;
    dA[14] = fma(dA[8], ux, A[8] * wx);
    A[15] = A[5] * ux;
    dA[15] = fma(dA[5], ux, A[5] * wx);
    A[16] = A[9] * uy;
    dA[16] = fma(dA[9], uy, A[9] * wy);
    A[17] = A[6] * ux;
    dA[17] = fma(dA[6], ux, A[6] * wx);
    A[18] = A[6] * uy;
    dA[18] = fma(dA[6], uy, A[6] * wy);
    A[19] = A[9] * ux;
    dA[19] = fma(dA[9], ux, A[9] * wx);
  }
  template <typename T>
  static __device__ __forceinline__ void grad(const T* e, const T* A, T& gx, T& gy, T& gz) {
    T g0 = T(0), g1 = T(0), g2 = T(0);
    g0 = fma(e[1], A[0], g0);
    g1 = fma(e[2], A[0], g1);
    g2 = fma(e[3], A[0], g2);
    g0 = fma(T(2) * e[4], A[1], g0);
    g1 = fma(T(2) * e[5], A[2], g1);
    g2 = fma(T(2) * e[6], A[3], g2);
    g0 = fma(e[7], A[2], g0);
    g1 = fma(e[7], A[1], g1);
    g0 = fma(e[8], A[3], g0);
    g2 = fma(e[8], A[1], g2);
    g1 = fma(e[9], A[3], g1);
    g2 = fma(e[9], A[2], g2);
    g0 = fma(T(3) * e[10], A[4], g0);
    g1 = fma(T(3) * e[11], A[5], g1);
    g2 = fma(T(3) * e[12], A[6], g2);
    g0 = fma(T(2) * e[13], A[7], g0);
    g1 = fma(e[13], A[4], g1);
    g0 = fma(T(2) * e[14], A[8], g0);
    g2 = fma(e[14], A[4], g2);
    g0 = fma(e[15], A[5], g0);
    g1 = fma(T(2) * e[15], A[7], g1);
    g1 = fma(T(2) * e[16], A[9], g1);
    g2 = fma(e[16], A[5], g2);
    g0 = fma(e[17], A[6], g0);
    g2 = fma(T(2) * e[17], A[8], g2);
    g1 = fma(e[18], A[6], g1);
    g2 = fma(T(2) * e[18], A[9], g2);
    g0 = fma(e[19], A[9], g0);
    g1 = fma(e[19], A[8], g1);
    g2 = fma(e[19], A[7], g2);
    gx = g0; gy = g1; gz = g2;
  }
  template <typename T>
  static __device__ __forceinline__ void dot_grad_deg(const T* e, const T* A, T* s, T* gx, T* gy, T* gz) {
    for (int n = 0; n <= 3; ++n) { s[n] = T(0); gx[n] = T(0); gy[n] = T(0); gz[n] = T(0); }
    s[0] = fma(e[0], A[0], s[0]);
    s[1] = fma(e[1], A[1], s[1]);
    gx[1] = fma(e[1], A[0], gx[1]);
    s[1] = fma(e[2], A[2], s[1]);
    gy[1] = fma(e[2], A[0], gy[1]);
    s[1] = fma(e[3], A[3], s[1]);
    gz[1] = fma(e[3], A[0], gz[1]);
    s[2] = fma(e[4], A[4], s[2]);
    gx[2] = fma(T(2) * e[4], A[1], gx[2]);
    s[2] = fma(e[5], A[5], s[2]);
    gy[2] = fma(T(2) * e[5], A[2], gy[2]);
    s[2] = fma(e[6], A[6], s[2]);
    gz[2] = fma(T(2) * e[6], A[3], gz[2]);
    s[2] = fma(e[7], A[7], s[2]);
    gx[2] = fma(e[7], A[2], gx[2]);
    gy[2] = fma(e[7], A[1], gy[2]);
    s[2] = fma(e[8], A[8], s[2]);
    gx[2] = fma(e[8], A[3], gx[2]);
    gz[2] = fma(e[8], A[1], gz[2]);
    s[2] = fma(e[9], A[9], s[2]);
    gy[2] = fma(e[9], A[3], gy[2]);
    gz[2] = fma(e[9], A[2], gz[2]);
    s[3] = fma(e[10], A[10], s[3]);
    gx[3] = fma(T(3) * e[10], A[4], gx[3]);
    s[3] = fma(e[11], A[11], s[3]);
    gy[3] = fma(T(3) * e[11], A[5], gy[3]);
    s[3] = fma(e[12], A[12], s[3]);
    gz[3] = fma(T(3) * e[12], A[6], gz[3]);
    s[3] = fma(e[13], A[13], s[3]);
    gx[3] = fma(T(2) * e[13], A[7], gx[3]);
    gy[3] = fma(e[13], A[4], gy[3]);
    s[3] = fma(e[14], A[14], s[3]);
    gx[3] = fma(T(2) * e[14], A[8], gx[3]);
    gz[3] = fma(e[14], A[4], gz[3]);
    s[3] = fma(e[15], A[15], s[3]);
    gx[3] = fma(e[15], A[5], gx[3]);
    gy[3] = fma(T(2) * e[15], A[7], gy[3]);
    s[3] = fma(e[16], A[16], s[3]);
    gy[3] = fma(T(2) * e[16], A[9], gy[3]);
    gz[3] = fma(e[16], A[5], gz[3]);
    s[3] = fma(e[17], A[17], s[3]);
    gx[3] = fma(e[17], A[6], gx[3]);
    gz[3] = fma(T(2) * e[17], A[8], gz[3]);
    s[3] = fma(e[18], A[18], s[3]);
    gy[3] = fma(e[18], A[6], gy[3]);
    gz[3] = fma(T(2) * e[18], A[9], gz[3]);
    s[3] = fma(e[19], A[19], s[3]);
    gx[3] = fma(e[19], A[9], gx[3]);
    gy[3] = fma(e[19], A[8], gy[3]);
    gz[3] = fma(e[19], A[7], gz[3]);
  }
  template <typename T>
  static __device__ __forceinline__ void d3(const T* B, T* d) {
    d[0] = B[0] * B[0];
    d[1] = B[1] * B[1] + B[2] * B[2] + B[3] * B[3];
    d[2] = B[4] * B[4] + B[5] * B[5] + B[6] * B[6] + T(2) * B[7] * B[7] + T(2) * B[8] * B[8] + T(2) * B[9] * B[9];
    d[3] = B[10] * B[10] + B[11] * B[11] + B[12] * B[12] + T(3) * B[13] * B[13] + T(3) * B[14] * B[14] + T(3) * B[15] * B[15] + T(3) * B[16] * B[16] + T(3) * B[17] * B[17] + T(3) * B[18] * B[18] + T(6) * B[19] * B[19];
  }
  template <typename T>
  static __device__ __forceinline__ void d3_tangent(const T* B, const T* Bd, T* d) {
    d[0] = T(2) * B[0] * Bd[0];
    d[1] = T(2) * B[1] * Bd[1] + T(2) * B[2] * Bd[2] + T(2) * B[3] * Bd[3];
    d[2] = T(2) * B[4] * Bd[4] + T(2) * B[5] * Bd[5] + T(2) * B[6] * Bd[6] + T(4) * B[7] * Bd[7] + T(4) * B[8] * Bd[8] + T(4) * B[9] * Bd[9];
    d[3] = T(2) * B[10] * Bd[10] + T(2) * B[11] * Bd[11] + T(2) * B[12] * Bd[12] + T(6) * B[13] * Bd[13] + T(6) * B[14] * Bd[14] + T(6) * B[15] * Bd[15] + T(6) * B[16] * Bd[16] + T(6) * B[17] * Bd[17] + T(6) * B[18] * Bd[18] + T(12) * B[19] * Bd[19];
  }
  template <typename T>
  static __device__ __forceinline__ void d3_adjoint(const T* B, const T* h, T* a) {
    a[0] = fma(T(2) * h[0], B[0], a[0]);
    a[1] = fma(T(2) * h[1], B[1], a[1]);
    a[2] = fma(T(2) * h[1], B[2], a[2]);
    a[3] = fma(T(2) * h[1], B[3], a[3]);
    a[4] = fma(T(2) * h[2], B[4], a[4]);
    a[5] = fma(T(2) * h[2], B[5], a[5]);
    a[6] = fma(T(2) * h[2], B[6], a[6]);
    a[7] = fma(T(4) * h[2], B[7], a[7]);
    a[8] = fma(T(4) * h[2], B[8], a[8]);
    a[9] = fma(T(4) * h[2], B[9], a[9]);
    a[10] = fma(T(2) * h[3], B[10], a[10]);
    a[11] = fma(T(2) * h[3], B[11], a[11]);
    a[12] = fma(T(2) * h[3], B[12], a[12]);
    a[13] = fma(T(6) * h[3], B[13], a[13]);
    a[14] = fma(T(6) * h[3], B[14], a[14]);
    a[15] = fma(T(6) * h[3], B[15], a[15]);
    a[16] = fma(T(6) * h[3], B[16], a[16]);
    a[17] = fma(T(6) * h[3], B[17], a[17]);
    a[18] = fma(T(6) * h[3], B[18], a[18]);
    a[19] = fma(T(12) * h[3], B[19], a[19]);
  }
};
template <> struct Four<3> {
  static constexpr int KA = 7;
  static __device__ __forceinline__ int p_n00(int n) {
    switch (n) {
      case 0: return 0;
      case 1: return 1;
      case 2: return 2;
      case 3: return 4;
      default: return -1;
    }
  }
  template <typename T>
  static __device__ __forceinline__ void desc(const T* B, const T* d3, T* D) {
    D[0] = B[0] * d3[0];
    D[1] = B[0] * d3[1];
    D[2] = B[0] * d3[2];
    D[3] = B[1] * B[1] * B[4] + T(2) * B[1] * B[2] * B[7] + T(2) * B[1] * B[3] * B[8] + B[2] * B[2] * B[5] + T(2) * B[2] * B[3] * B[9] + B[3] * B[3] * B[6];
    D[4] = B[0] * d3[3];
    D[5] = B[1] * B[4] * B[10] + B[2] * B[4] * B[13] + B[3] * B[4] * B[14] + B[1] * B[5] * B[15] + B[2] * B[5] * B[11] + B[3] * B[5] * B[16] + B[1] * B[6] * B[17] + B[2] * B[6] * B[18] + B[3] * B[6] * B[12] + T(2) * B[1] * B[7] * B[13] + T(2) * B[2] * B[7] * B[15] + T(2) * B[3] * B[7] * B[19] + T(2) * B[1] * B[8] * B[14] + T(2) * B[2] * B[8] * B[19] + T(2) * B[3] * B[8] * B[17] + T(2) * B[1] * B[9] * B[19] + T(2) * B[2] * B[9] * B[16] + T(2) * B[3] * B[9] * B[18];
    D[6] = B[4] * B[4] * B[4] + T(3) * B[4] * B[7] * B[7] + T(3) * B[4] * B[8] * B[8] + T(3) * B[5] * B[7] * B[7] + T(6) * B[7] * B[8] * B[9] + T(3) * B[6] * B[8] * B[8] + B[5] * B[5] * B[5] + T(3) * B[5] * B[9] * B[9] + T(3) * B[6] * B[9] * B[9] + B[6] * B[6] * B[6];
  }
  template <typename T>
  static __device__ __forceinline__ void adjoint(const T* B, const T* w, T* a) {
    {
      const T wp = w[3];
      a[1] = fma(wp, B[1] * B[4], a[1]);
      a[1] = fma(wp, B[1] * B[4], a[1]);
      a[4] = fma(wp, B[1] * B[1], a[4]);
      const T wk1_2_7 = T(2) * wp;
      a[1] = fma(wk1_2_7, B[2] * B[7], a[1]);
      a[2] = fma(wk1_2_7, B[1] * B[7], a[2]);
      a[7] = fma(wk1_2_7, B[1] * B[2], a[7]);
      const T wk1_3_8 = T(2) * wp;
      a[1] = fma(wk1_3_8, B[3] * B[8], a[1]);
      a[3] = fma(wk1_3_8, B[1] * B[8], a[3]);
      a[8] = fma(wk1_3_8, B[1] * B[3], a[8]);
      a[2] = fma(wp, B[2] * B[5], a[2]);
      a[2] = fma(wp, B[2] * B[5], a[2]);
      a[5] = fma(wp, B[2] * B[2], a[5]);
      const T wk2_3_9 = T(2) * wp;
      a[2] = fma(wk2_3_9, B[3] * B[9], a[2]);
      a[3] = fma(wk2_3_9, B[2] * B[9], a[3]);
      a[9] = fma(wk2_3_9, B[2] * B[3], a[9]);
      a[3] = fma(wp, B[3] * B[6], a[3]);
      a[3] = fma(wp, B[3] * B[6], a[3]);
      a[6] = fma(wp, B[3] * B[3], a[6]);
    }
    {
      const T wp = w[5];
      a[1] = fma(wp, B[4] * B[10], a[1]);
      a[4] = fma(wp, B[1] * B[10], a[4]);
      a[10] = fma(wp, B[1] * B[4], a[10]);
      a[2] = fma(wp, B[4] * B[13], a[2]);
      a[4] = fma(wp, B[2] * B[13], a[4]);
      a[13] = fma(wp, B[2] * B[4], a[13]);
      a[3] = fma(wp, B[4] * B[14], a[3]);
      a[4] = fma(wp, B[3] * B[14], a[4]);
      a[14] = fma(wp, B[3] * B[4], a[14]);
      a[1] = fma(wp, B[5] * B[15], a[1]);
      a[5] = fma(wp, B[1] * B[15], a[5]);
      a[15] = fma(wp, B[1] * B[5], a[15]);
      a[2] = fma(wp, B[5] * B[11], a[2]);
      a[5] = fma(wp, B[2] * B[11], a[5]);
      a[11] = fma(wp, B[2] * B[5], a[11]);
      a[3] = fma(wp, B[5] * B[16], a[3]);
      a[5] = fma(wp, B[3] * B[16], a[5]);
      a[16] = fma(wp, B[3] * B[5], a[16]);
      a[1] = fma(wp, B[6] * B[17], a[1]);
      a[6] = fma(wp, B[1] * B[17], a[6]);
      a[17] = fma(wp, B[1] * B[6], a[17]);
      a[2] = fma(wp, B[6] * B[18], a[2]);
      a[6] = fma(wp, B[2] * B[18], a[6]);
      a[18] = fma(wp, B[2] * B[6], a[18]);
      a[3] = fma(wp, B[6] * B[12], a[3]);
      a[6] = fma(wp, B[3] * B[12], a[6]);
      a[12] = fma(wp, B[3] * B[6], a[12]);
      const T wk1_7_13 = T(2) * wp;
      a[1] = fma(wk1_7_13, B[7] * B[13], a[1]);
      a[7] = fma(wk1_7_13, B[1] * B[13], a[7]);
      a[13] = fma(wk1_7_13, B[1] * B[7], a[13]);
      const T wk2_7_15 = T(2) * wp;
      a[2] = fma(wk2_7_15, B[7] * B[15], a[2]);
      a[7] = fma(wk2_7_15, B[2] * B[15], a[7]);
      a[15] = fma(wk2_7_15, B[2] * B[7], a[15]);
      const T wk3_7_19 = T(2) * wp;
      a[3] = fma(wk3_7_19, B[7] * B[19], a[3]);
      a[7] = fma(wk3_7_19, B[3] * B[19], a[7]);
      a[19] = fma(wk3_7_19, B[3] * B[7], a[19]);
      const T wk1_8_14 = T(2) * wp;
      a[1] = fma(wk1_8_14, B[8] * B[14], a[1]);
      a[8] = fma(wk1_8_14, B[1] * B[14], a[8]);
      a[14] = fma(wk1_8_14, B[1] * B[8], a[14]);
      const T wk2_8_19 = T(2) * wp;
      a[2] = fma(wk2_8_19, B[8] * B[19], a[2]);
      a[8] = fma(wk2_8_19, B[2] * B[19], a[8]);
      a[19] = fma(wk2_8_19, B[2] * B[8], a[19]);
      const T wk3_8_17 = T(2) * wp;
      a[3] = fma(wk3_8_17, B[8] * B[17], a[3]);
      a[8] = fma(wk3_8_17, B[3] * B[17], a[8]);
      a[17] = fma(wk3_8_17, B[3] * B[8], a[17]);
      const T wk1_9_19 = T(2) * wp;
      a[1] = fma(wk1_9_19, B[9] * B[19], a[1]);
      a[9] = fma(wk1_9_19, B[1] * B[19], a[9]);
      a[19] = fma(wk1_9_19, B[1] * B[9], a[19]);
      const T wk2_9_16 = T(2) * wp;
      a[2] = fma(wk2_9_16, B[9] * B[16], a[2]);
      a[9] = fma(wk2_9_16, B[2] * B[16], a[9]);
      a[16] = fma(wk2_9_16, B[2] * B[9], a[16]);
      const T wk3_9_18 = T(2) * wp;
      a[3] = fma(wk3_9_18, B[9] * B[18], a[3]);
      a[9] = fma(wk3_9_18, B[3] * B[18], a[9]);
      a[18] = fma(wk3_9_18, B[3] * B[9], a[18]);
    }
    {
      const T wp = w[6];
      a[4] = fma(wp, B[4] * B[4], a[4]);
      a[4] = fma(wp, B[4] * B[4], a[4]);
      a[4] = fma(wp, B[4] * B[4], a[4]);
      const T wk4_7_7 = T(3) * wp;
      a[4] = fma(wk4_7_7, B[7] * B[7], a[4]);
      a[7] = fma(wk4_7_7, B[4] * B[7], a[7]);
      a[7] = fma(wk4_7_7, B[4] * B[7], a[7]);
      const T wk4_8_8 = T(3) * wp;
      a[4] = fma(wk4_8_8, B[8] * B[8], a[4]);
      a[8] = fma(wk4_8_8, B[4] * B[8], a[8]);
      a[8] = fma(wk4_8_8, B[4] * B[8], a[8]);
      const T wk5_7_7 = T(3) * wp;
      a[5] = fma(wk5_7_7, B[7] * B[7], a[5]);
      a[7] = fma(wk5_7_7, B[5] * B[7], a[7]);
      a[7] = fma(wk5_7_7, B[5] * B[7], a[7]);
      const T wk7_8_9 = T(6) * wp;
      a[7] = fma(wk7_8_9, B[8] * B[9], a[7]);
      a[8] = fma(wk7_8_9, B[7] * B[9], a[8]);
      a[9] = fma(wk7_8_9, B[7] * B[8], a[9]);
      const T wk6_8_8 = T(3) * wp;
      a[6] = fma(wk6_8_8, B[8] * B[8], a[6]);
      a[8] = fma(wk6_8_8, B[6] * B[8], a[8]);
      a[8] = fma(wk6_8_8, B[6] * B[8], a[8]);
      a[5] = fma(wp, B[5] * B[5], a[5]);
      a[5] = fma(wp, B[5] * B[5], a[5]);
      a[5] = fma(wp, B[5] * B[5], a[5]);
      const T wk5_9_9 = T(3) * wp;
      a[5] = fma(wk5_9_9, B[9] * B[9], a[5]);
      a[9] = fma(wk5_9_9, B[5] * B[9], a[9]);
      a[9] = fma(wk5_9_9, B[5] * B[9], a[9]);
      const T wk6_9_9 = T(3) * wp;
      a[6] = fma(wk6_9_9, B[9] * B[9], a[6]);
      a[9] = fma(wk6_9_9, B[6] * B[9], a[9]);
      a[9] = fma(wk6_9_9, B[6] * B[9], a[9]);
      a[6] = fma(wp, B[6] * B[6], a[6]);
      a[6] = fma(wp, B[6] * B[6], a[6]);
      a[6] = fma(wp, B[6] * B[6], a[6]);
    }
  }
  template <typename T>
  static __device__ __forceinline__ void tangent(const T* B, const T* Bd, const T* d3, const T* d3d, T* Dd) {
    Dd[0] = fma(Bd[0], d3[0], B[0] * d3d[0]);
    Dd[1] = fma(Bd[0], d3[1], B[0] * d3d[1]);
    Dd[2] = fma(Bd[0], d3[2], B[0] * d3d[2]);
    Dd[3] = (Bd[1] * B[1] * B[4] + B[1] * Bd[1] * B[4] + B[1] * B[1] * Bd[4]) + T(2) * (Bd[1] * B[2] * B[7] + B[1] * Bd[2] * B[7] + B[1] * B[2] * Bd[7]) + T(2) * (Bd[1] * B[3] * B[8] + B[1] * Bd[3] * B[8] + B[1] * B[3] * Bd[8]) + (Bd[2] * B[2] * B[5] + B[2] * Bd[2] * B[5] + B[2] * B[2] * Bd[5]) + T(2) * (Bd[2] * B[3] * B[9] + B[2] * Bd[3] * B[9] + B[2] * B[3] * Bd[9]) + (Bd[3] * B[3] * B[6] + B[3] * Bd[3] * B[6] + B[3] * B[3] * Bd[6]);
    Dd[4] = fma(Bd[0], d3[3], B[0] * d3d[3]);
    Dd[5] = (Bd[1] * B[4] * B[10] + B[1] * Bd[4] * B[10] + B[1] * B[4] * Bd[10]) + (Bd[2] * B[4] * B[13] + B[2] * Bd[4] * B[13] + B[2] * B[4] * Bd[13]) + (Bd[3] * B[4] * B[14] + B[3] * Bd[4] * B[14] + B[3] * B[4] * Bd[14]) + (Bd[1] * B[5] * B[15] + B[1] * Bd[5] * B[15] + B[1] * B[5] * Bd[15]) + (Bd[2] * B[5] * B[11] + B[2] * Bd[5] * B[11] + B[2] * B[5] * Bd[11]) + (Bd[3] * B[5] * B[16] + B[3] * Bd[5] * B[16] + B[3] * B[5] * Bd[16]) + (Bd[1] * B[6] * B[17] + B[1] * Bd[6] * B[17] + B[1] * B[6] * Bd[17]) + (Bd[2] * B[6] * B[18] + B[2] * Bd[6] * B[18] + B[2] * B[6] * Bd[18]) + (Bd[3] * B[6] * B[12] + B[3] * Bd[6] * B[12] + B[3] * B[6] * Bd[12]) + T(2) * (Bd[1] * B[7] * B[13] + B[1] * Bd[7] * B[13] + B[1] * B[7] * Bd[13]) + T(2) * (Bd[2] * B[7] * B[15] + B[2] * Bd[7] * B[15] + B[2] * B[7] * Bd[15]) + T(2) * (Bd[3] * B[7] * B[19] + B[3] * Bd[7] * B[19] + B[3] * B[7] * Bd[19]) + T(2) * (Bd[1] * B[8] * B[14] + B[1] * Bd[8] * B[14] + B[1] * B[8] * Bd[14]) + T(2) * (Bd[2] * B[8] * B[19] + B[2] * Bd[8] * B[19] + B[2] * B[8] * Bd[19]) + T(2) * (Bd[3] * B[8] * B[17] + B[3] * Bd[8] * B[17] + B[3] * B[8] * Bd[17]) + T(2) * (Bd[1] * B[9] * B[19] + B[1] * Bd[9] * B[19] + B[1] * B[9] * Bd[19]) + T(2) * (Bd[2] * B[9] * B[16] + B[2] * Bd[9] * B[16] + B[2] * B[9] * Bd[16]) + T(2) * (Bd[3] * B[9] * B[18] + B[3] * Bd[9] * B[18] + B[3] * B[9] * Bd[18]);
    Dd[6] = (Bd[4] * B[4] * B[4] + B[4] * Bd[4] * B[4] + B[4] * B[4] * Bd[4]) + T(3) * (Bd[4] * B[7] * B[7] + B[4] * Bd[7] * B[7] + B[4] * B[7] * Bd[7]) + T(3) * (Bd[4] * B[8] * B[8] + B[4] * Bd[8] * B[8] + B[4] * B[8] * Bd[8]) + T(3) * (Bd[5] * B[7] * B[7] + B[5] * Bd[7] * B[7] + B[5] * B[7] * Bd[7]) + T(6) * (Bd[7] * B[8] * B[9] + B[7] * Bd[8] * B[9] + B[7] * B[8] * Bd[9]) + T(3) * (Bd[6] * B[8] * B[8] + B[6] * Bd[8] * B[8] + B[6] * B[8] * Bd[8]) + (Bd[5] * B[5] * B[5] + B[5] * Bd[5] * B[5] + B[5] * B[5] * Bd[5]) + T(3) * (Bd[5] * B[9] * B[9] + B[5] * Bd[9] * B[9] + B[5] * B[9] * Bd[9]) + T(3) * (Bd[6] * B[9] * B[9] + B[6] * Bd[9] * B[9] + B[6] * B[9] * Bd[9]) + (Bd[6] * B[6] * B[6] + B[6] * Bd[6] * B[6] + B[6] * B[6] * Bd[6]);
  }
  static constexpr int NTERMS = 34;
};
template <> struct Mono<4> {
  static constexpr int NA = 35;
  template <typename T>
  static __device__ __forceinline__ void eval(T ux, T uy, T uz, T* A) {
    A[0] = T(1);
    A[1] = ux;
    A[2] = uy;
    A[3] = uz;
    A[4] = A[1] * ux;
    A[5] = A[2] * uy;
    A[6] = A[3] * uz;
    A[7] = A[2] * ux;
    A[8] = A[3] * ux;
    A[9] = A[3] * uy;
    A[10] = A[4] * ux;
    A[11] = A[5] * uy;
    A[12] = A[6] * uz;
    A[13] = A[7] * ux;
    A[14] = A[8] * ux;
    A[15] = A[5] * ux;
    A[16] = A[9] * uy;
    A[17] = A[6] * ux;
    A[18] = A[6] * uy;
    A[19] = A[9] * ux;
    A[20] = A[10] * ux;
    A[21] = A[11] * uy;
    A[22] = A[12] * uz;
    A[23] = A[13] * ux;
    A[24] = A[14] * ux;
    A[25] = A[11] * ux;
    A[26] = A[16] * uy;
    A[27] = A[12] * ux;
    A[28] = A[12] * uy;
    A[29] = A[15] * ux;
    A[30] = A[17] * ux;
    A[31] = A[18] * uy;
    A[32] = A[19] * ux;
    A[33] = A[16] * ux;
    A[34] = A[18] * ux;
  }
  static constexpr int NA2 = 18;
  static __device__ __forceinline__ void eval2(float ux, float uy, float uz, float2* A2) {
    A2[0].x = 1.0f;
    A2[0].y = ux;
    A2[1].x = uy;
    A2[1].y = uz;
    A2[2].x = A2[0].y * ux;
    A2[2].y = A2[1].x * uy;
    A2[3].x = A2[1].y * uz;
    A2[3].y = A2[1].x * ux;
    A2[4].x = A2[1].y * ux;
    A2[4].y = A2[1].y * uy;
    A2[5].x = A2[2].x * ux;
    A2[5].y = A2[2].y * uy;
    A2[6].x = A2[3].x * uz;
    A2[6].y = A2[3].y * ux;
    A2[7].x = A2[4].x * ux;
    A2[7].y = A2[2].y * ux;
    A2[8].x = A2[4].y * uy;
    A2[8].y = A2[3].x * ux;
    A2[9].x = A2[3].x * uy;
    A2[9].y = A2[4].y * ux;
    A2[10].x = A2[5].x * ux;
    A2[10].y = A2[5].y * uy;
    A2[11].x = A2[6].x * uz;
    A2[11].y = A2[6].y * ux;
    A2[12].x = A2[7].x * ux;
    A2[12].y = A2[5].y * ux;
    A2[13].x = A2[8].x * uy;
    A2[13].y = A2[6].x * ux;
    A2[14].x = A2[6].x * uy;
    A2[14].y = A2[7].y * ux;
    A2[15].x = A2[8].y * ux;
    A2[15].y = A2[9].x * uy;
    A2[16].x = A2[9].y * ux;
    A2[16].y = A2[8].x * ux;
    A2[17].x = A2[9].x * ux;
    A2[17].y = 0.0f;
  }
  template <typename T>
  static __device__ __forceinline__ void eval_d(T ux, T uy, T uz, T wx, T wy, T wz, T* A, T* dA) {
    A[0] = T(1);
    dA[0] = T(0);
    A[1] = ux;
    dA[1] = wx;
    A[2] = uy;
    dA[2] = wy;
    A[3] = uz;
    dA[3] = wz;
    A[4] = A[1] * ux;
    dA[4] = fma(dA[1], ux, A[1] * wx);
    A[5] = A[2] * uy;
    dA[5] = fma(dA[2], uy, A[2] * wy);
    A[6] = A[3] * uz;
    dA[6] = fma(dA[3], uz, A[3] * wz);
    A[7] = A[2] * ux;
    dA[7] = fma(dA[2], ux, A[2] * wx);
    A[8] = A[3] * ux;
    dA[8] = fma(dA[3], ux, A[3] * wx);
    A[9] = A[3] * uy;
    dA[9] = fma(dA[3], uy, A[3] * wy);
    A[10] = A[4] * ux;
    dA[10] = fma(dA[4], ux, A[4] * wx);
    A[11] = A[5] * uy;
    dA[11] = fma(dA[5], uy, A[5] * wy);
    A[12] = A[6] * uz;
    dA[12] = fma(dA[6], uz, A[6] * wz);
    A[13] = A[7] * ux;
    dA[13] = fma(dA[7], ux, A[7] * wx);
    A[14] = A[8] * ux;
    dA[14] = fma(dA[8], ux, A[8] * wx);
    A[15] = A[5] * ux;
    dA[15] = fma(dA[5], ux, A[5] * wx);
    A[16] = A[9] * uy;
    dA[16] = fma(dA[9], uy, A[9] * wy);
    A[17] = A[6] * ux;
    dA[17] = fma(dA[6], ux, A[6] * wx);
    A[18] = A[6] * uy;
    dA[18] = fma(dA[6], uy, A[6] * wy);
    A[19] = A[9] * ux;
    dA[19] = fma(dA[9], ux, A[9] * wx);
    A[20] = A[10] * ux;
    dA[20] = fma(dA[10], ux, A[10] * wx);
    A[21] = A[11] * uy;
    dA[21] = fma(dA[11], uy, A[11] * wy);
    A[22] = A[12] * uz;
    dA[22] = fma(dA[12], uz, A[12] * wz);
    A[23] = A[13] * ux;
    dA[23] = fma(dA[13], ux, A[13] * wx);
    A[24] = A[14] * ux;
    dA[24] = fma(dA[14], ux, A[14] * wx);
    A[25] = A[11] * ux;
    dA[25] = fma(dA[11], ux, A[11] * wx);
    A[26] = A[16] * uy;
    dA[26] = fma(dA[16], uy, A[16] * wy);
    A[27] = A[12] * ux;
    dA[27] = fma(dA[12], ux, A[12] * wx);
    A[28] = A[12] * uy;
    dA[28] = fma(dA[12], uy, A[12] * wy);
    A[29] = A[15] * ux;
    dA[29] = fma(dA[15], ux, A[15] * wx);
    A[30] = A[17] * ux;
    dA[30] = fma(dA[17], ux, A[17] * wx);
    A[31] = A[18] * uy;
    dA[31] = fma(dA[18], uy, A[18] * wy);
    A[32] = A[19] * ux;
    dA[32] = fma(dA[19], ux, A[19] * wx);
    A[33] = A[16] * ux;
    dA[33] = fma(dA[16], ux, A[16] * wx);
    A[34] = A[18] * ux;
    dA[34] = fma(dA[18], ux, A[18] * wx);
  }
  template <typename T>
  static __device__ __forceinline__ void grad(const T* e, const T* A, T& gx, T& gy, T& gz) {
    T g0 = T(0), g1 = T(0), g2 = T(0);
    g0 = fma(e[1], A[0], g0);
    g1 = fma(e[2], A[0], g1);
    g2 = fma(e[3], A[0], g2);
    g0 = fma(T(2) * e[4], A[1], g0);
    g1 = fma(T(2) * e[5], A[2], g1);
    g2 = fma(T(2) * e[6], A[3], g2);
    g0 = fma(e[7], A[2], g0);
    g1 = fma(e[7], A[1], g1);
    g0 = fma(e[8], A[3], g0);
    g2 = fma(e[8], A[1], g2);
    g1 = fma(e[9], A[3], g1);
    g2 = fma(e[9], A[2], g2);
    g0 = fma(T(3) * e[10], A[4], g0);
    g1 = fma(T(3) * e[11], A[5], g1);
    g2 = fma(T(3) * e[12], A[6], g2);
    g0 = fma(T(2) * e[13], A[7], g0);
    g1 = fma(e[13], A[4], g1);
    g0 = fma(T(2) * e[14], A[8], g0);
    g2 = fma(e[14], A[4], g2);
    g0 = fma(e[15], A[5], g0);
    g1 = fma(T(2) * e[15], A[7], g1);
    g1 = fma(T(2) * e[16], A[9], g1);
    g2 = fma(e[16], A[5], g2);
    g0 = fma(e[17], A[6], g0);
    g2 = fma(T(2) * e[17], A[8], g2);
    g1 = fma(e[18], A[6], g1);
    g2 = fma(T(2) * e[18], A[9], g2);
    g0 = fma(e[19], A[9], g0);
    g1 = fma(e[19], A[8], g1);
    g2 = fma(e[19], A[7], g2);
    g0 = fma(T(4) * e[20], A[10], g0);
    g1 = fma(T(4) * e[21], A[11], g1);
    g2 = fma(T(4) * e[22], A[12], g2);
    g0 = fma(T(3) * e[23], A[13], g0);
    g1 = fma(e[23], A[10], g1);
    g0 = fma(T(3) * e[24], A[14], g0);
    g2 = fma(e[24], A[10], g2);
    g0 = fma(e[25], A[11], g0);
    g1 = fma(T(3) * e[25], A[15], g1);
    g1 = fma(T(3) * e[26], A[16], g1);
    g2 = fma(e[26], A[11], g2);
    g0 = fma(e[27], A[12], g0);
    g2 = fma(T(3) * e[27], A[17], g2);
    g1 = fma(e[28], A[12], g1);
    g2 = fma(T(3) * e[28], A[18], g2);
    g0 = fma(T(2) * e[29], A[15], g0);
    g1 = fma(T(2) * e[29], A[13], g1);
    g0 = fma(T(2) * e[30], A[17], g0);
    g2 = fma(T(2) * e[30], A[14], g2);
    g1 = fma(T(2) * e[31], A[18], g1);
    g2 = fma(T(2) * e[31], A[16], g2);
    g0 = fma(T(2) * e[32], A[19], g0);
    g1 = fma(e[32], A[14], g1);
    g2 = fma(e[32], A[13], g2);
    g0 = fma(e[33], A[16], g0);
    g1 = fma(T(2) * e[33], A[19], g1);
    g2 = fma(e[33], A[15], g2);
    g0 = fma(e[34], A[18], g0);
    g1 = fma(e[34], A[17], g1);
    g2 = fma(T(2) * e[34], A[19], g2);
    gx = g0; gy = g1; gz = g2;
  }
  template <typename T>
  static __device__ __forceinline__ void dot_grad_deg(const T* e, const T* A, T* s, T* gx, T* gy, T* gz) {
    for (int n = 0; n <= 4; ++n) { s[n] = T(0); gx[n] = T(0); gy[n] = T(0); gz[n] = T(0); }
    s[0] = fma(e[0], A[0], s[0]);
    s[1] = fma(e[1], A[1], s[1]);
    gx[1] = fma(e[1], A[0], gx[1]);
    s[1] = fma(e[2], A[2], s[1]);
    gy[1] = fma(e[2], A[0], gy[1]);
    s[1] = fma(e[3], A[3], s[1]);
    gz[1] = fma(e[3], A[0], gz[1]);
    s[2] = fma(e[4], A[4], s[2]);
    gx[2] = fma(T(2) * e[4], A[1], gx[2]);
    s[2] = fma(e[5], A[5], s[2]);
    gy[2] = fma(T(2) * e[5], A[2], gy[2]);
    s[2] = fma(e[6], A[6], s[2]);
    gz[2] = fma(T(2) * e[6], A[3], gz[2]);
    s[2] = fma(e[7], A[7], s[2]);
    gx[2] = fma(e[7], A[2], gx[2]);
    gy[2] = fma(e[7], A[1], gy[2]);
    s[2] = fma(e[8], A[8], s[2]);
    gx[2] = fma(e[8], A[3], gx[2]);
    gz[2] = fma(e[8], A[1], gz[2]);
    s[2] = fma(e[9], A[9], s[2]);
    gy[2] = fma(e[9], A[3], gy[2]);
    gz[2] = fma(e[9], A[2], gz[2]);
    s[3] = fma(e[10], A[10], s[3]);
    gx[3] = fma(T(3) * e[10], A[4], gx[3]);
    s[3] = fma(e[11], A[11], s[3]);
    gy[3] = fma(T(3) * e[11], A[5], gy[3]);
    s[3] = fma(e[12], A[12], s[3]);
    gz[3] = fma(T(3) * e[12], A[6], gz[3]);
    s[3] = fma(e[13], A[13], s[3]);
    gx[3] = fma(T(2) * e[13], A[7], gx[3]);
    gy[3] = fma(e[13], A[4], gy[3]);
    s[3] = fma(e[14], A[14], s[3]);
    gx[3] = fma(T(2) * e[14], A[8], gx[3]);
    gz[3] = fma(e[14], A[4], gz[3]);
    s[3] = fma(e[15], A[15], s[3]);
    gx[3] = fma(e[15], A[5], gx[3]);
    gy[3] = fma(T(2) * e[15], A[7], gy[3]);
    s[3] = fma(e[16], A[16], s[3]);
    gy[3] = fma(T(2) * e[16], A[9], gy[3]);
    gz[3] = fma(e[16], A[5], gz[3]);
    s[3] = fma(e[17], A[17], s[3]);
    gx[3] = fma(e[17], A[6], gx[3]);
    gz[3] = fma(T(2) * e[17], A[8], gz[3]);
    s[3] = fma(e[18], A[18], s[3]);
    gy[3] = fma(e[18], A[6], gy[3]);
    gz[3] = fma(T(2) * e[18], A[9], gz[3]);
    s[3] = fma(e[19], A[19], s[3]);
    gx[3] = fma(e[19], A[9], gx[3]);
    gy[3] = fma(e[19], A[8], gy[3]);
    gz[3] = fma(e[19], A[7], gz[3]);
    s[4] = fma(e[20], A[20], s[4]);
    gx[4] = fma(T(4) * e[20], A[10], gx[4]);
    s[4] = fma(e[21], A[21], s[4]);
    gy[4] = fma(T(4) * e[21], A[11], gy[4]);
    s[4] = fma(e[22], A[22], s[4]);
    gz[4] = fma(T(4) * e[22], A[12], gz[4]);
    s[4] = fma(e[23], A[23], s[4]);
    gx[4] = fma(T(3) * e[23], A[13], gx[4]);
    gy[4] = fma(e[23], A[10], gy[4]);
    s[4] = fma(e[24], A[24], s[4]);
    gx[4] = fma(T(3) * e[24], A[14], gx[4]);
    gz[4] = fma(e[24], A[10], gz[4]);
    s[4] = fma(e[25], A[25], s[4]);
    gx[4] = fma(e[25], A[11], gx[4]);
    gy[4] = fma(T(3) * e[25], A[15], gy[4]);
    s[4] = fma(e[26], A[26], s[4]);
    gy[4] = fma(T(3) * e[26], A[16], gy[4]);
    gz[4] = fma(e[26], A[11], gz[4]);
    s[4] = fma(e[27], A[27], s[4]);
    gx[4] = fma(e[27], A[12], gx[4]);
    gz[4] = fma(T(3) * e[27], A[17], gz[4]);
    s[4] = fma(e[28], A[28], s[4]);
    gy[4] = fma(e[28], A[12], gy[4]);
    gz[4] = fma(T(3) * e[28], A[18], gz[4]);
    s[4] = fma(e[29], A[29], s[4]);
    gx[4] = fma(T(2) * e[29], A[15], gx[4]);
    gy[4] = fma(T(2) * e[29], A[13], gy[4]);
    s[4] = fma(e[30], A[30], s[4]);
    gx[4] = fma(T(2) * e[30], A[17], gx[4]);
    gz[4] = fma(T(2) * e[30], A[14], gz[4]);
    s[4] = fma(e[31], A[31], s[4]);
    gy[4] = fma(T(2) * e[31], A[18], gy[4]);
    gz[4] = fma(T(2) * e[31], A[16], gz[4]);
    s[4] = fma(e[32], A[32], s[4]);
    gx[4] = fma(T(2) * e[32], A[19], gx[4]);
    gy[4] = fma(e[32], A[14], gy[4]);
    gz[4] = fma(e[32], A[13], gz[4]);
    s[4] = fma(e[33], A[33], s[4]);
    gx[4] = fma(e[33], A[16], gx[4]);
    gy[4] = fma(T(2) * e[33], A[19], gy[4]);
    gz[4] = fma(e[33], A[15], gz[4]);
    s[4] = fma(e[34], A[34], s[4]);
    gx[4] = fma(e[34], A[18], gx[4]);
    gy[4] = fma(e[34], A[17], gy[4]);
    gz[4] = fma(T(2) * e[34], A[19], gz[4]);
  }
  template <typename T>
  static __device__ __forceinline__ void d3(const T* B, T* d) {
    d[0] = B[0] * B[0];
    d[1] = B[1] * B[1] + B[2] * B[2] + B[3] * B[3];
    d[2] = B[4] * B[4] + B[5] * B[5] + B[6] * B[6] + T(2) * B[7] * B[7] + T(2) * B[8] * B[8] + T(2) * B[9] * B[9];
    d[3] = B[10] * B[10] + B[11] * B[11] + B[12] * B[12] + T(3) * B[13] * B[13] + T(3) * B[14] * B[14] + T(3) * B[15] * B[15] + T(3) * B[16] * B[16] + T(3) * B[17] * B[17] + T(3) * B[18] * B[18] + T(6) * B[19] * B[19];
    d[4] = B[20] * B[20] + B[21] * B[21] + B[22] * B[22] + T(4) * B[23] * B[23] + T(4) * B[24] * B[24] + T(4) * B[25] * B[25] + T(4) * B[26] * B[26] + T(4) * B[27] * B[27] + T(4) * B[28] * B[28] + T(6) * B[29] * B[29] + T(6) * B[30] * B[30] + T(6) * B[31] * B[31] + T(12) * B[32] * B[32] + T(12) * B[33] * B[33] + T(12) * B[34] * B[34];
  }
  template <typename T>
  static __device__ __forceinline__ void d3_tangent(const T* B, const T* Bd, T* d) {
    d[0] = T(2) * B[0] * Bd[0];
    d[1] = T(2) * B[1] * Bd[1] + T(2) * B[2] * Bd[2] + T(2) * B[3] * Bd[3];
    d[2] = T(2) * B[4] * Bd[4] + T(2) * B[5] * Bd[5] + T(2) * B[6] * Bd[6] + T(4) * B[7] * Bd[7] + T(4) * B[8] * Bd[8] + T(4) * B[9] * Bd[9];
    d[3] = T(2) * B[10] * Bd[10] + T(2) * B[11] * Bd[11] + T(2) * B[12] * Bd[12] + T(6) * B[13] * Bd[13] + T(6) * B[14] * Bd[14] + T(6) * B[15] * Bd[15] + T(6) * B[16] * Bd[16] + T(6) * B[17] * Bd[17] + T(6) * B[18] * Bd[18] + T(12) * B[19] * Bd[19];
    d[4] = T(2) * B[20] * Bd[20] + T(2) * B[21] * Bd[21] + T(2) * B[22] * Bd[22] + T(8) * B[23] * Bd[23] + T(8) * B[24] * Bd[24] + T(8) * B[25] * Bd[25] + T(8) * B[26] * Bd[26] + T(8) * B[27] * Bd[27] + T(8) * B[28] * Bd[28] + T(12) * B[29] * Bd[29] + T(12) * B[30] * Bd[30] + T(12) * B[31] * Bd[31] + T(24) * B[32] * Bd[32] + T(24) * B[33] * Bd[33] + T(24) * B[34] * Bd[34];
  }
  template <typename T>
  static __device__ __forceinline__ void d3_adjoint(const T* B, const T* h, T* a) {
    a[0] = fma(T(2) * h[0], B[0], a[0]);
    a[1] = fma(T(2) * h[1], B[1], a[1]);
    a[2] = fma(T(2) * h[1], B[2], a[2]);
    a[3] = fma(T(2) * h[1], B[3], a[3]);
    a[4] = fma(T(2) * h[2], B[4], a[4]);
    a[5] = fma(T(2) * h[2], B[5], a[5]);
    a[6] = fma(T(2) * h[2], B[6], a[6]);
    a[7] = fma(T(4) * h[2], B[7], a[7]);
    a[8] = fma(T(4) * h[2], B[8], a[8]);
    a[9] = fma(T(4) * h[2], B[9], a[9]);
    a[10] = fma(T(2) * h[3], B[10], a[10]);
    a[11] = fma(T(2) * h[3], B[11], a[11]);
    a[12] = fma(T(2) * h[3], B[12], a[12]);
    a[13] = fma(T(6) * h[3], B[13], a[13]);
    a[14] = fma(T(6) * h[3], B[14], a[14]);
    a[15] = fma(T(6) * h[3], B[15], a[15]);
    a[16] = fma(T(6) * h[3], B[16], a[16]);
    a[17] = fma(T(6) * h[3], B[17], a[17]);
    a[18] = fma(T(6) * h[3], B[18], a[18]);
    a[19] = fma(T(12) * h[3], B[19], a[19]);
    a[20] = fma(T(2) * h[4], B[20], a[20]);
    a[21] = fma(T(2) * h[4], B[21], a[21]);
    a[22] = fma(T(2) * h[4], B[22], a[22]);
    a[23] = fma(T(8) * h[4], B[23], a[23]);
    a[24] = fma(T(8) * h[4], B[24], a[24]);
    a[25] = fma(T(8) * h[4], B[25], a[25]);
    a[26] = fma(T(8) * h[4], B[26], a[26]);
    a[27] = fma(T(8) * h[4], B[27], a[27]);
    a[28] = fma(T(8) * h[4], B[28], a[28]);
    a[29] = fma(T(12) * h[4], B[29], a[29]);
    a[30] = fma(T(12) * h[4], B[30], a[30]);
    a[31] = fma(T(12) * h[4], B[31], a[31]);
    a[32] = fma(T(24) * h[4], B[32], a[32]);
    a[33] = fma(T(24) * h[4], B[33], a[33]);
    a[34] = fma(T(24) * h[4], B[34], a[34]);
  }
};
template <> struct Four<4> {
  static constexpr int KA = 11;
  static __device__ __forceinline__ int p_n00(int n) {
    switch (n) {
      case 0: return 0;
      case 1: return 1;
      case 2: return 2;
      case 3: return 4;
      case 4: return 7;
      default: return -1;
    }
  }
  template <typename T>
  static __device__ __forceinline__ void desc(const T* B, const T* d3, T* D) {
    D[0] = B[0] * d3[0];
    D[1] = B[0] * d3[1];
    D[2] = B[0] * d3[2];
    D[3] = B[1] * B[1] * B[4] + T(2) * B[1] * B[2] * B[7] + T(2) * B[1] * B[3] * B[8] + B[2] * B[2] * B[5] + T(2) * B[2] * B[3] * B[9] + B[3] * B[3] * B[6];
    D[4] = B[0] * d3[3];
    D[5] = B[1] * B[4] * B[10] + B[2] * B[4] * B[13] + B[3] * B[4] * B[14] + B[1] * B[5] * B[15] + B[2] * B[5] * B[11] + B[3] * B[5] * B[16] + B[1] * B[6] * B[17] + B[2] * B[6] * B[18] + B[3] * B[6] * B[12] + T(2) * B[1] * B[7] * B[13] + T(2) * B[2] * B[7] * B[15] + T(2) * B[3] * B[7] * B[19] + T(2) * B[1] * B[8] * B[14] + T(2) * B[2] * B[8] * B[19] + T(2) * B[3] * B[8] * B[17] + T(2) * B[1] * B[9] * B[19] + T(2) * B[2] * B[9] * B[16] + T(2) * B[3] * B[9] * B[18];
    D[6] = B[4] * B[4] * B[4] + T(3) * B[4] * B[7] * B[7] + T(3) * B[4] * B[8] * B[8] + T(3) * B[5] * B[7] * B[7] + T(6) * B[7] * B[8] * B[9] + T(3) * B[6] * B[8] * B[8] + B[5] * B[5] * B[5] + T(3) * B[5] * B[9] * B[9] + T(3) * B[6] * B[9] * B[9] + B[6] * B[6] * B[6];
    D[7] = B[0] * d3[4];
    D[8] = B[1] * B[10] * B[20] + B[2] * B[10] * B[23] + B[3] * B[10] * B[24] + B[1] * B[11] * B[25] + B[2] * B[11] * B[21] + B[3] * B[11] * B[26] + B[1] * B[12] * B[27] + B[2] * B[12] * B[28] + B[3] * B[12] * B[22] + T(3) * B[1] * B[13] * B[23] + T(3) * B[2] * B[13] * B[29] + T(3) * B[3] * B[13] * B[32] + T(3) * B[1] * B[14] * B[24] + T(3) * B[2] * B[14] * B[32] + T(3) * B[3] * B[14] * B[30] + T(3) * B[1] * B[15] * B[29] + T(3) * B[2] * B[15] * B[25] + T(3) * B[3] * B[15] * B[33] + T(3) * B[1] * B[16] * B[33] + T(3) * B[2] * B[16] * B[26] + T(3) * B[3] * B[16] * B[31] + T(3) * B[1] * B[17] * B[30] + T(3) * B[2] * B[17] * B[34] + T(3) * B[3] * B[17] * B[27] + T(3) * B[1] * B[18] * B[34] + T(3) * B[2] * B[18] * B[31] + T(3) * B[3] * B[18] * B[28] + T(6) * B[1] * B[19] * B[32] + T(6) * B[2] * B[19] * B[33] + T(6) * B[3] * B[19] * B[34];
    D[9] = B[4] * B[4] * B[20] + T(2) * B[4] * B[5] * B[29] + T(2) * B[4] * B[6] * B[30] + T(4) * B[4] * B[7] * B[23] + T(4) * B[4] * B[8] * B[24] + T(4) * B[4] * B[9] * B[32] + B[5] * B[5] * B[21] + T(2) * B[5] * B[6] * B[31] + T(4) * B[5] * B[7] * B[25] + T(4) * B[5] * B[8] * B[33] + T(4) * B[5] * B[9] * B[26] + B[6] * B[6] * B[22] + T(4) * B[6] * B[7] * B[34] + T(4) * B[6] * B[8] * B[27] + T(4) * B[6] * B[9] * B[28] + T(4) * B[7] * B[7] * B[29] + T(8) * B[7] * B[8] * B[32] + T(8) * B[7] * B[9] * B[33] + T(4) * B[8] * B[8] * B[30] + T(8) * B[8] * B[9] * B[34] + T(4) * B[9] * B[9] * B[31];
    D[10] = B[4] * B[10] * B[10] + T(2) * B[7] * B[10] * B[13] + T(2) * B[8] * B[10] * B[14] + B[5] * B[13] * B[13] + T(2) * B[9] * B[13] * B[14] + B[6] * B[14] * B[14] + B[4] * B[15] * B[15] + T(2) * B[7] * B[11] * B[15] + T(2) * B[8] * B[15] * B[16] + B[5] * B[11] * B[11] + T(2) * B[9] * B[11] * B[16] + B[6] * B[16] * B[16] + B[4] * B[17] * B[17] + T(2) * B[7] * B[17] * B[18] + T(2) * B[8] * B[12] * B[17] + B[5] * B[18] * B[18] + T(2) * B[9] * B[12] * B[18] + B[6] * B[12] * B[12] + T(2) * B[4] * B[13] * B[13] + T(4) * B[7] * B[13] * B[15] + T(4) * B[8] * B[13] * B[19] + T(2) * B[5] * B[15] * B[15] + T(4) * B[9] * B[15] * B[19] + T(2) * B[6] * B[19] * B[19] + T(2) * B[4] * B[14] * B[14] + T(4) * B[7] * B[14] * B[19] + T(4) * B[8] * B[14] * B[17] + T(2) * B[5] * B[19] * B[19] + T(4) * B[9] * B[17] * B[19] + T(2) * B[6] * B[17] * B[17] + T(2) * B[4] * B[19] * B[19] + T(4) * B[7] * B[16] * B[19] + T(4) * B[8] * B[18] * B[19] + T(2) * B[5] * B[16] * B[16] + T(4) * B[9] * B[16] * B[18] + T(2) * B[6] * B[18] * B[18];
  }
  template <typename T>
  static __device__ __forceinline__ void adjoint(const T* B, const T* w, T* a) {
    {
      const T wp = w[3];
      a[1] = fma(wp, B[1] * B[4], a[1]);
      a[1] = fma(wp, B[1] * B[4], a[1]);
      a[4] = fma(wp, B[1] * B[1], a[4]);
      const T wk1_2_7 = T(2) * wp;
      a[1] = fma(wk1_2_7, B[2] * B[7], a[1]);
      a[2] = fma(wk1_2_7, B[1] * B[7], a[2]);
      a[7] = fma(wk1_2_7, B[1] * B[2], a[7]);
      const T wk1_3_8 = T(2) * wp;
      a[1] = fma(wk1_3_8, B[3] * B[8], a[1]);
      a[3] = fma(wk1_3_8, B[1] * B[8], a[3]);
      a[8] = fma(wk1_3_8, B[1] * B[3], a[8]);
      a[2] = fma(wp, B[2] * B[5], a[2]);
      a[2] = fma(wp, B[2] * B[5], a[2]);
      a[5] = fma(wp, B[2] * B[2], a[5]);
      const T wk2_3_9 = T(2) * wp;
      a[2] = fma(wk2_3_9, B[3] * B[9], a[2]);
      a[3] = fma(wk2_3_9, B[2] * B[9], a[3]);
      a[9] = fma(wk2_3_9, B[2] * B[3], a[9]);
      a[3] = fma(wp, B[3] * B[6], a[3]);
      a[3] = fma(wp, B[3] * B[6], a[3]);
      a[6] = fma(wp, B[3] * B[3], a[6]);
    }
    {
      const T wp = w[5];
      a[1] = fma(wp, B[4] * B[10], a[1]);
      a[4] = fma(wp, B[1] * B[10], a[4]);
      a[10] = fma(wp, B[1] * B[4], a[10]);
      a[2] = fma(wp, B[4] * B[13], a[2]);
      a[4] = fma(wp, B[2] * B[13], a[4]);
      a[13] = fma(wp, B[2] * B[4], a[13]);
      a[3] = fma(wp, B[4] * B[14], a[3]);
      a[4] = fma(wp, B[3] * B[14], a[4]);
      a[14] = fma(wp, B[3] * B[4], a[14]);
      a[1] = fma(wp, B[5] * B[15], a[1]);
      a[5] = fma(wp, B[1] * B[15], a[5]);
      a[15] = fma(wp, B[1] * B[5], a[15]);
      a[2] = fma(wp, B[5] * B[11], a[2]);
      a[5] = fma(wp, B[2] * B[11], a[5]);
      a[11] = fma(wp, B[2] * B[5], a[11]);
      a[3] = fma(wp, B[5] * B[16], a[3]);
      a[5] = fma(wp, B[3] * B[16], a[5]);
      a[16] = fma(wp, B[3] * B[5], a[16]);
      a[1] = fma(wp, B[6] * B[17], a[1]);
      a[6] = fma(wp, B[1] * B[17], a[6]);
      a[17] = fma(wp, B[1] * B[6], a[17]);
      a[2] = fma(wp, B[6] * B[18], a[2]);
      a[6] = fma(wp, B[2] * B[18], a[6]);
      a[18] = fma(wp, B[2] * B[6], a[18]);
      a[3] = fma(wp, B[6] * B[12], a[3]);
      a[6] = fma(wp, B[3] * B[12], a[6]);
      a[12] = fma(wp, B[3] * B[6], a[12]);
      const T wk1_7_13 = T(2) * wp;
      a[1] = fma(wk1_7_13, B[7] * B[13], a[1]);
      a[7] = fma(wk1_7_13, B[1] * B[13], a[7]);
      a[13] = fma(wk1_7_13, B[1] * B[7], a[13]);
      const T wk2_7_15 = T(2) * wp;
      a[2] = fma(wk2_7_15, B[7] * B[15], a[2]);
      a[7] = fma(wk2_7_15, B[2] * B[15], a[7]);
      a[15] = fma(wk2_7_15, B[2] * B[7], a[15]);
      const T wk3_7_19 = T(2) * wp;
      a[3] = fma(wk3_7_19, B[7] * B[19], a[3]);
      a[7] = fma(wk3_7_19, B[3] * B[19], a[7]);
      a[19] = fma(wk3_7_19, B[3] * B[7], a[19]);
      const T wk1_8_14 = T(2) * wp;
      a[1] = fma(wk1_8_14, B[8] * B[14], a[1]);
      a[8] = fma(wk1_8_14, B[1] * B[14], a[8]);
      a[14] = fma(wk1_8_14, B[1] * B[8], a[14]);
      const T wk2_8_19 = T(2) * wp;
      a[2] = fma(wk2_8_19, B[8] * B[19], a[2]);
      a[8] = fma(wk2_8_19, B[2] * B[19], a[8]);
      a[19] = fma(wk2_8_19, B[2] * B[8], a[19]);
      const T wk3_8_17 = T(2) * wp;
      a[3] = fma(wk3_8_17, B[8] * B[17], a[3]);
      a[8] = fma(wk3_8_17, B[3] * B[17], a[8]);
      a[17] = fma(wk3_8_17, B[3] * B[8], a[17]);
      const T wk1_9_19 = T(2) * wp;
      a[1] = fma(wk1_9_19, B[9] * B[19], a[1]);
      a[9] = fma(wk1_9_19, B[1] * B[19], a[9]);
      a[19] = fma(wk1_9_19, B[1] * B[9], a[19]);
      const T wk2_9_16 = T(2) * wp;
      a[2] = fma(wk2_9_16, B[9] * B[16], a[2]);
      a[9] = fma(wk2_9_16, B[2] * B[16], a[9]);
      a[16] = fma(wk2_9_16, B[2] * B[9], a[16]);
      const T wk3_9_18 = T(2) * wp;
      a[3] = fma(wk3_9_18, B[9] * B[18], a[3]);
      a[9] = fma(wk3_9_18, B[3] * B[18], a[9]);
      a[18] = fma(wk3_9_18, B[3] * B[9], a[18]);
    }
    {
      const T wp = w[6];
      a[4] = fma(wp, B[4] * B[4], a[4]);
      a[4] = fma(wp, B[4] * B[4], a[4]);
      a[4] = fma(wp, B[4] * B[4], a[4]);
      const T wk4_7_7 = T(3) * wp;
      a[4] = fma(wk4_7_7, B[7] * B[7], a[4]);
      a[7] = fma(wk4_7_7, B[4] * B[7], a[7]);
      a[7] = fma(wk4_7_7, B[4] * B[7], a[7]);
      const T wk4_8_8 = T(3) * wp;
      a[4] = fma(wk4_8_8, B[8] * B[8], a[4]);
      a[8] = fma(wk4_8_8, B[4] * B[8], a[8]);
      a[8] = fma(wk4_8_8, B[4] * B[8], a[8]);
      const T wk5_7_7 = T(3) * wp;
      a[5] = fma(wk5_7_7, B[7] * B[7], a[5]);
      a[7] = fma(wk5_7_7, B[5] * B[7], a[7]);
      a[7] = fma(wk5_7_7, B[5] * B[7], a[7]);
      const T wk7_8_9 = T(6) * wp;
      a[7] = fma(wk7_8_9, B[8] * B[9], a[7]);
      a[8] = fma(wk7_8_9, B[7] * B[9], a[8]);
      a[9] = fma(wk7_8_9, B[7] * B[8], a[9]);
      const T wk6_8_8 = T(3) * wp;
      a[6] = fma(wk6_8_8, B[8] * B[8], a[6]);
      a[8] = fma(wk6_8_8, B[6] * B[8], a[8]);
      a[8] = fma(wk6_8_8, B[6] * B[8], a[8]);
      a[5] = fma(wp, B[5] * B[5], a[5]);
      a[5] = fma(wp, B[5] * B[5], a[5]);
      a[5] = fma(wp, B[5] * B[5], a[5]);
      const T wk5_9_9 = T(3) * wp;
      a[5] = fma(wk5_9_9, B[9] * B[9], a[5]);
      a[9] = fma(wk5_9_9, B[5] * B[9], a[9]);
      a[9] = fma(wk5_9_9, B[5] * B[9], a[9]);
      const T wk6_9_9 = T(3) * wp;
      a[6] = fma(wk6_9_9, B[9] * B[9], a[6]);
      a[9] = fma(wk6_9_9, B[6] * B[9], a[9]);
      a[9] = fma(wk6_9_9, B[6] * B[9], a[9]);
      a[6] = fma(wp, B[6] * B[6], a[6]);
      a[6] = fma(wp, B[6] * B[6], a[6]);
      a[6] = fma(wp, B[6] * B[6], a[6]);
    }
    {
      const T wp = w[8];
      a[1] = fma(wp, B[10] * B[20], a[1]);
      a[10] = fma(wp, B[1] * B[20], a[10]);
      a[20] = fma(wp, B[1] * B[10], a[20]);
      a[2] = fma(wp, B[10] * B[23], a[2]);
      a[10] = fma(wp, B[2] * B[23], a[10]);
      a[23] = fma(wp, B[2] * B[10], a[23]);
      a[3] = fma(wp, B[10] * B[24], a[3]);
      a[10] = fma(wp, B[3] * B[24], a[10]);
      a[24] = fma(wp, B[3] * B[10], a[24]);
      a[1] = fma(wp, B[11] * B[25], a[1]);
      a[11] = fma(wp, B[1] * B[25], a[11]);
      a[25] = fma(wp, B[1] * B[11], a[25]);
      a[2] = fma(wp, B[11] * B[21], a[2]);
      a[11] = fma(wp, B[2] * B[21], a[11]);
      a[21] = fma(wp, B[2] * B[11], a[21]);
      a[3] = fma(wp, B[11] * B[26], a[3]);
      a[11] = fma(wp, B[3] * B[26], a[11]);
      a[26] = fma(wp, B[3] * B[11], a[26]);
      a[1] = fma(wp, B[12] * B[27], a[1]);
      a[12] = fma(wp, B[1] * B[27], a[12]);
      a[27] = fma(wp, B[1] * B[12], a[27]);
      a[2] = fma(wp, B[12] * B[28], a[2]);
      a[12] = fma(wp, B[2] * B[28], a[12]);
      a[28] = fma(wp, B[2] * B[12], a[28]);
      a[3] = fma(wp, B[12] * B[22], a[3]);
      a[12] = fma(wp, B[3] * B[22], a[12]);
      a[22] = fma(wp, B[3] * B[12], a[22]);
      const T wk1_13_23 = T(3) * wp;
      a[1] = fma(wk1_13_23, B[13] * B[23], a[1]);
      a[13] = fma(wk1_13_23, B[1] * B[23], a[13]);
      a[23] = fma(wk1_13_23, B[1] * B[13], a[23]);
      const T wk2_13_29 = T(3) * wp;
      a[2] = fma(wk2_13_29, B[13] * B[29], a[2]);
      a[13] = fma(wk2_13_29, B[2] * B[29], a[13]);
      a[29] = fma(wk2_13_29, B[2] * B[13], a[29]);
      const T wk3_13_32 = T(3) * wp;
      a[3] = fma(wk3_13_32, B[13] * B[32], a[3]);
      a[13] = fma(wk3_13_32, B[3] * B[32], a[13]);
      a[32] = fma(wk3_13_32, B[3] * B[13], a[32]);
      const T wk1_14_24 = T(3) * wp;
      a[1] = fma(wk1_14_24, B[14] * B[24], a[1]);
      a[14] = fma(wk1_14_24, B[1] * B[24], a[14]);
      a[24] = fma(wk1_14_24, B[1] * B[14], a[24]);
      const T wk2_14_32 = T(3) * wp;
      a[2] = fma(wk2_14_32, B[14] * B[32], a[2]);
      a[14] = fma(wk2_14_32, B[2] * B[32], a[14]);
      a[32] = fma(wk2_14_32, B[2] * B[14], a[32]);
      const T wk3_14_30 = T(3) * wp;
      a[3] = fma(wk3_14_30, B[14] * B[30], a[3]);
      a[14] = fma(wk3_14_30, B[3] * B[30], a[14]);
      a[30] = fma(wk3_14_30, B[3] * B[14], a[30]);
      const T wk1_15_29 = T(3) * wp;
      a[1] = fma(wk1_15_29, B[15] * B[29], a[1]);
      a[15] = fma(wk1_15_29, B[1] * B[29], a[15]);
      a[29] = fma(wk1_15_29, B[1] * B[15], a[29]);
      const T wk2_15_25 = T(3) * wp;
      a[2] = fma(wk2_15_25, B[15] * B[25], a[2]);
      a[15] = fma(wk2_15_25, B[2] * B[25], a[15]);
      a[25] = fma(wk2_15_25, B[2] * B[15], a[25]);
      const T wk3_15_33 = T(3) * wp;
      a[3] = fma(wk3_15_33, B[15] * B[33], a[3]);
      a[15] = fma(wk3_15_33, B[3] * B[33], a[15]);
      a[33] = fma(wk3_15_33, B[3] * B[15], a[33]);
      const T wk1_16_33 = T(3) * wp;
      a[1] = fma(wk1_16_33, B[16] * B[33], a[1]);
      a[16] = fma(wk1_16_33, B[1] * B[33], a[16]);
      a[33] = fma(wk1_16_33, B[1] * B[16], a[33]);
      const T wk2_16_26 = T(3) * wp;
      a[2] = fma(wk2_16_26, B[16] * B[26], a[2]);
      a[16] = fma(wk2_16_26, B[2] * B[26], a[16]);
      a[26] = fma(wk2_16_26, B[2] * B[16], a[26]);
      const T wk3_16_31 = T(3) * wp;
      a[3] = fma(wk3_16_31, B[16] * B[31], a[3]);
      a[16] = fma(wk3_16_31, B[3] * B[31], a[16]);
      a[31] = fma(wk3_16_31, B[3] * B[16], a[31]);
      const T wk1_17_30 = T(3) * wp;
      a[1] = fma(wk1_17_30, B[17] * B[30], a[1]);
      a[17] = fma(wk1_17_30, B[1] * B[30], a[17]);
      a[30] = fma(wk1_17_30, B[1] * B[17], a[30]);
      const T wk2_17_34 = T(3) * wp;
      a[2] = fma(wk2_17_34, B[17] * B[34], a[2]);
      a[17] = fma(wk2_17_34, B[2] * B[34], a[17]);
      a[34] = fma(wk2_17_34, B[2] * B[17], a[34]);
      const T wk3_17_27 = T(3) * wp;
      a[3] = fma(wk3_17_27, B[17] * B[27], a[3]);
      a[17] = fma(wk3_17_27, B[3] * B[27], a[17]);
      a[27] = fma(wk3_17_27, B[3] * B[17], a[27]);
      const T wk1_18_34 = T(3) * wp;
      a[1] = fma(wk1_18_34, B[18] * B[34], a[1]);
      a[18] = fma(wk1_18_34, B[1] * B[34], a[18]);
      a[34] = fma(wk1_18_34, B[1] * B[18], a[34]);
      const T wk2_18_31 = T(3) * wp;
      a[2] = fma(wk2_18_31, B[18] * B[31], a[2]);
      a[18] = fma(wk2_18_31, B[2] * B[31], a[18]);
      a[31] = fma(wk2_18_31, B[2] * B[18], a[31]);
      const T wk3_18_28 = T(3) * wp;
      a[3] = fma(wk3_18_28, B[18] * B[28], a[3]);
      a[18] = fma(wk3_18_28, B[3] * B[28], a[18]);
      a[28] = fma(wk3_18_28, B[3] * B[18], a[28]);
      const T wk1_19_32 = T(6) * wp;
      a[1] = fma(wk1_19_32, B[19] * B[32], a[1]);
      a[19] = fma(wk1_19_32, B[1] * B[32], a[19]);
      a[32] = fma(wk1_19_32, B[1] * B[19], a[32]);
      const T wk2_19_33 = T(6) * wp;
      a[2] = fma(wk2_19_33, B[19] * B[33], a[2]);
      a[19] = fma(wk2_19_33, B[2] * B[33], a[19]);
      a[33] = fma(wk2_19_33, B[2] * B[19], a[33]);
      const T wk3_19_34 = T(6) * wp;
      a[3] = fma(wk3_19_34, B[19] * B[34], a[3]);
      a[19] = fma(wk3_19_34, B[3] * B[34], a[19]);
      a[34] = fma(wk3_19_34, B[3] * B[19], a[34]);
    }
    {
      const T wp = w[9];
      a[4] = fma(wp, B[4] * B[20], a[4]);
      a[4] = fma(wp, B[4] * B[20], a[4]);
      a[20] = fma(wp, B[4] * B[4], a[20]);
      const T wk4_5_29 = T(2) * wp;
      a[4] = fma(wk4_5_29, B[5] * B[29], a[4]);
      a[5] = fma(wk4_5_29, B[4] * B[29], a[5]);
      a[29] = fma(wk4_5_29, B[4] * B[5], a[29]);
      const T wk4_6_30 = T(2) * wp;
      a[4] = fma(wk4_6_30, B[6] * B[30], a[4]);
      a[6] = fma(wk4_6_30, B[4] * B[30], a[6]);
      a[30] = fma(wk4_6_30, B[4] * B[6], a[30]);
      const T wk4_7_23 = T(4) * wp;
      a[4] = fma(wk4_7_23, B[7] * B[23], a[4]);
      a[7] = fma(wk4_7_23, B[4] * B[23], a[7]);
      a[23] = fma(wk4_7_23, B[4] * B[7], a[23]);
      const T wk4_8_24 = T(4) * wp;
      a[4] = fma(wk4_8_24, B[8] * B[24], a[4]);
      a[8] = fma(wk4_8_24, B[4] * B[24], a[8]);
      a[24] = fma(wk4_8_24, B[4] * B[8], a[24]);
      const T wk4_9_32 = T(4) * wp;
      a[4] = fma(wk4_9_32, B[9] * B[32], a[4]);
      a[9] = fma(wk4_9_32, B[4] * B[32], a[9]);
      a[32] = fma(wk4_9_32, B[4] * B[9], a[32]);
      a[5] = fma(wp, B[5] * B[21], a[5]);
      a[5] = fma(wp, B[5] * B[21], a[5]);
      a[21] = fma(wp, B[5] * B[5], a[21]);
      const T wk5_6_31 = T(2) * wp;
      a[5] = fma(wk5_6_31, B[6] * B[31], a[5]);
      a[6] = fma(wk5_6_31, B[5] * B[31], a[6]);
      a[31] = fma(wk5_6_31, B[5] * B[6], a[31]);
      const T wk5_7_25 = T(4) * wp;
      a[5] = fma(wk5_7_25, B[7] * B[25], a[5]);
      a[7] = fma(wk5_7_25, B[5] * B[25], a[7]);
      a[25] = fma(wk5_7_25, B[5] * B[7], a[25]);
      const T wk5_8_33 = T(4) * wp;
      a[5] = fma(wk5_8_33, B[8] * B[33], a[5]);
      a[8] = fma(wk5_8_33, B[5] * B[33], a[8]);
      a[33] = fma(wk5_8_33, B[5] * B[8], a[33]);
      const T wk5_9_26 = T(4) * wp;
      a[5] = fma(wk5_9_26, B[9] * B[26], a[5]);
      a[9] = fma(wk5_9_26, B[5] * B[26], a[9]);
      a[26] = fma(wk5_9_26, B[5] * B[9], a[26]);
      a[6] = fma(wp, B[6] * B[22], a[6]);
      a[6] = fma(wp, B[6] * B[22], a[6]);
      a[22] = fma(wp, B[6] * B[6], a[22]);
      const T wk6_7_34 = T(4) * wp;
      a[6] = fma(wk6_7_34, B[7] * B[34], a[6]);
      a[7] = fma(wk6_7_34, B[6] * B[34], a[7]);
      a[34] = fma(wk6_7_34, B[6] * B[7], a[34]);
      const T wk6_8_27 = T(4) * wp;
      a[6] = fma(wk6_8_27, B[8] * B[27], a[6]);
      a[8] = fma(wk6_8_27, B[6] * B[27], a[8]);
      a[27] = fma(wk6_8_27, B[6] * B[8], a[27]);
      const T wk6_9_28 = T(4) * wp;
      a[6] = fma(wk6_9_28, B[9] * B[28], a[6]);
      a[9] = fma(wk6_9_28, B[6] * B[28], a[9]);
      a[28] = fma(wk6_9_28, B[6] * B[9], a[28]);
      const T wk7_7_29 = T(4) * wp;
      a[7] = fma(wk7_7_29, B[7] * B[29], a[7]);
      a[7] = fma(wk7_7_29, B[7] * B[29], a[7]);
      a[29] = fma(wk7_7_29, B[7] * B[7], a[29]);
      const T wk7_8_32 = T(8) * wp;
      a[7] = fma(wk7_8_32, B[8] * B[32], a[7]);
      a[8] = fma(wk7_8_32, B[7] * B[32], a[8]);
      a[32] = fma(wk7_8_32, B[7] * B[8], a[32]);
      const T wk7_9_33 = T(8) * wp;
      a[7] = fma(wk7_9_33, B[9] * B[33], a[7]);
      a[9] = fma(wk7_9_33, B[7] * B[33], a[9]);
      a[33] = fma(wk7_9_33, B[7] * B[9], a[33]);
      const T wk8_8_30 = T(4) * wp;
      a[8] = fma(wk8_8_30, B[8] * B[30], a[8]);
      a[8] = fma(wk8_8_30, B[8] * B[30], a[8]);
      a[30] = fma(wk8_8_30, B[8] * B[8], a[30]);
      const T wk8_9_34 = T(8) * wp;
      a[8] = fma(wk8_9_34, B[9] * B[34], a[8]);
      a[9] = fma(wk8_9_34, B[8] * B[34], a[9]);
      a[34] = fma(wk8_9_34, B[8] * B[9], a[34]);
      const T wk9_9_31 = T(4) * wp;
      a[9] = fma(wk9_9_31, B[9] * B[31], a[9]);
      a[9] = fma(wk9_9_31, B[9] * B[31], a[9]);
      a[31] = fma(wk9_9_31, B[9] * B[9], a[31]);
    }
    {
      const T wp = w[10];
      a[4] = fma(wp, B[10] * B[10], a[4]);
      a[10] = fma(wp, B[4] * B[10], a[10]);
      a[10] = fma(wp, B[4] * B[10], a[10]);
      const T wk7_10_13 = T(2) * wp;
      a[7] = fma(wk7_10_13, B[10] * B[13], a[7]);
      a[10] = fma(wk7_10_13, B[7] * B[13], a[10]);
      a[13] = fma(wk7_10_13, B[7] * B[10], a[13]);
      const T wk8_10_14 = T(2) * wp;
      a[8] = fma(wk8_10_14, B[10] * B[14], a[8]);
      a[10] = fma(wk8_10_14, B[8] * B[14], a[10]);
      a[14] = fma(wk8_10_14, B[8] * B[10], a[14]);
      a[5] = fma(wp, B[13] * B[13], a[5]);
      a[13] = fma(wp, B[5] * B[13], a[13]);
      a[13] = fma(wp, B[5] * B[13], a[13]);
      const T wk9_13_14 = T(2) * wp;
      a[9] = fma(wk9_13_14, B[13] * B[14], a[9]);
      a[13] = fma(wk9_13_14, B[9] * B[14], a[13]);
      a[14] = fma(wk9_13_14, B[9] * B[13], a[14]);
      a[6] = fma(wp, B[14] * B[14], a[6]);
      a[14] = fma(wp, B[6] * B[14], a[14]);
      a[14] = fma(wp, B[6] * B[14], a[14]);
      a[4] = fma(wp, B[15] * B[15], a[4]);
      a[15] = fma(wp, B[4] * B[15], a[15]);
      a[15] = fma(wp, B[4] * B[15], a[15]);
      const T wk7_11_15 = T(2) * wp;
      a[7] = fma(wk7_11_15, B[11] * B[15], a[7]);
      a[11] = fma(wk7_11_15, B[7] * B[15], a[11]);
      a[15] = fma(wk7_11_15, B[7] * B[11], a[15]);
      const T wk8_15_16 = T(2) * wp;
      a[8] = fma(wk8_15_16, B[15] * B[16], a[8]);
      a[15] = fma(wk8_15_16, B[8] * B[16], a[15]);
      a[16] = fma(wk8_15_16, B[8] * B[15], a[16]);
      a[5] = fma(wp, B[11] * B[11], a[5]);
      a[11] = fma(wp, B[5] * B[11], a[11]);
      a[11] = fma(wp, B[5] * B[11], a[11]);
      const T wk9_11_16 = T(2) * wp;
      a[9] = fma(wk9_11_16, B[11] * B[16], a[9]);
      a[11] = fma(wk9_11_16, B[9] * B[16], a[11]);
      a[16] = fma(wk9_11_16, B[9] * B[11], a[16]);
      a[6] = fma(wp, B[16] * B[16], a[6]);
      a[16] = fma(wp, B[6] * B[16], a[16]);
      a[16] = fma(wp, B[6] * B[16], a[16]);
      a[4] = fma(wp, B[17] * B[17], a[4]);
      a[17] = fma(wp, B[4] * B[17], a[17]);
      a[17] = fma(wp, B[4] * B[17], a[17]);
      const T wk7_17_18 = T(2) * wp;
      a[7] = fma(wk7_17_18, B[17] * B[18], a[7]);
      a[17] = fma(wk7_17_18, B[7] * B[18], a[17]);
      a[18] = fma(wk7_17_18, B[7] * B[17], a[18]);
      const T wk8_12_17 = T(2) * wp;
      a[8] = fma(wk8_12_17, B[12] * B[17], a[8]);
      a[12] = fma(wk8_12_17, B[8] * B[17], a[12]);
      a[17] = fma(wk8_12_17, B[8] * B[12], a[17]);
      a[5] = fma(wp, B[18] * B[18], a[5]);
      a[18] = fma(wp, B[5] * B[18], a[18]);
      a[18] = fma(wp, B[5] * B[18], a[18]);
      const T wk9_12_18 = T(2) * wp;
      a[9] = fma(wk9_12_18, B[12] * B[18], a[9]);
      a[12] = fma(wk9_12_18, B[9] * B[18], a[12]);
      a[18] = fma(wk9_12_18, B[9] * B[12], a[18]);
      a[6] = fma(wp, B[12] * B[12], a[6]);
      a[12] = fma(wp, B[6] * B[12], a[12]);
      a[12] = fma(wp, B[6] * B[12], a[12]);
      const T wk4_13_13 = T(2) * wp;
      a[4] = fma(wk4_13_13, B[13] * B[13], a[4]);
      a[13] = fma(wk4_13_13, B[4] * B[13], a[13]);
      a[13] = fma(wk4_13_13, B[4] * B[13], a[13]);
      const T wk7_13_15 = T(4) * wp;
      a[7] = fma(wk7_13_15, B[13] * B[15], a[7]);
      a[13] = fma(wk7_13_15, B[7] * B[15], a[13]);
      a[15] = fma(wk7_13_15, B[7] * B[13], a[15]);
      const T wk8_13_19 = T(4) * wp;
      a[8] = fma(wk8_13_19, B[13] * B[19], a[8]);
      a[13] = fma(wk8_13_19, B[8] * B[19], a[13]);
      a[19] = fma(wk8_13_19, B[8] * B[13], a[19]);
      const T wk5_15_15 = T(2) * wp;
      a[5] = fma(wk5_15_15, B[15] * B[15], a[5]);
      a[15] = fma(wk5_15_15, B[5] * B[15], a[15]);
      a[15] = fma(wk5_15_15, B[5] * B[15], a[15]);
      const T wk9_15_19 = T(4) * wp;
      a[9] = fma(wk9_15_19, B[15] * B[19], a[9]);
      a[15] = fma(wk9_15_19, B[9] * B[19], a[15]);
      a[19] = fma(wk9_15_19, B[9] * B[15], a[19]);
      const T wk6_19_19 = T(2) * wp;
      a[6] = fma(wk6_19_19, B[19] * B[19], a[6]);
      a[19] = fma(wk6_19_19, B[6] * B[19], a[19]);
      a[19] = fma(wk6_19_19, B[6] * B[19], a[19]);
      const T wk4_14_14 = T(2) * wp;
      a[4] = fma(wk4_14_14, B[14] * B[14], a[4]);
      a[14] = fma(wk4_14_14, B[4] * B[14], a[14]);
      a[14] = fma(wk4_14_14, B[4] * B[14], a[14]);
      const T wk7_14_19 = T(4) * wp;
      a[7] = fma(wk7_14_19, B[14] * B[19], a[7]);
      a[14] = fma(wk7_14_19, B[7] * B[19], a[14]);
      a[19] = fma(wk7_14_19, B[7] * B[14], a[19]);
      const T wk8_14_17 = T(4) * wp;
      a[8] = fma(wk8_14_17, B[14] * B[17], a[8]);
      a[14] = fma(wk8_14_17, B[8] * B[17], a[14]);
      a[17] = fma(wk8_14_17, B[8] * B[14], a[17]);
      const T wk5_19_19 = T(2) * wp;
      a[5] = fma(wk5_19_19, B[19] * B[19], a[5]);
      a[19] = fma(wk5_19_19, B[5] * B[19], a[19]);
      a[19] = fma(wk5_19_19, B[5] * B[19], a[19]);
      const T wk9_17_19 = T(4) * wp;
      a[9] = fma(wk9_17_19, B[17] * B[19], a[9]);
      a[17] = fma(wk9_17_19, B[9] * B[19], a[17]);
      a[19] = fma(wk9_17_19, B[9] * B[17], a[19]);
      const T wk6_17_17 = T(2) * wp;
      a[6] = fma(wk6_17_17, B[17] * B[17], a[6]);
      a[17] = fma(wk6_17_17, B[6] * B[17], a[17]);
      a[17] = fma(wk6_17_17, B[6] * B[17], a[17]);
      const T wk4_19_19 = T(2) * wp;
      a[4] = fma(wk4_19_19, B[19] * B[19], a[4]);
      a[19] = fma(wk4_19_19, B[4] * B[19], a[19]);
      a[19] = fma(wk4_19_19, B[4] * B[19], a[19]);
      const T wk7_16_19 = T(4) * wp;
      a[7] = fma(wk7_16_19, B[16] * B[19], a[7]);
      a[16] = fma(wk7_16_19, B[7] * B[19], a[16]);
      a[19] = fma(wk7_16_19, B[7] * B[16], a[19]);
      const T wk8_18_19 = T(4) * wp;
      a[8] = fma(wk8_18_19, B[18] * B[19], a[8]);
      a[18] = fma(wk8_18_19, B[8] * B[19], a[18]);
      a[19] = fma(wk8_18_19, B[8] * B[18], a[19]);
      const T wk5_16_16 = T(2) * wp;
      a[5] = fma(wk5_16_16, B[16] * B[16], a[5]);
      a[16] = fma(wk5_16_16, B[5] * B[16], a[16]);
      a[16] = fma(wk5_16_16, B[5] * B[16], a[16]);
      const T wk9_16_18 = T(4) * wp;
      a[9] = fma(wk9_16_18, B[16] * B[18], a[9]);
      a[16] = fma(wk9_16_18, B[9] * B[18], a[16]);
      a[18] = fma(wk9_16_18, B[9] * B[16], a[18]);
      const T wk6_18_18 = T(2) * wp;
      a[6] = fma(wk6_18_18, B[18] * B[18], a[6]);
      a[18] = fma(wk6_18_18, B[6] * B[18], a[18]);
      a[18] = fma(wk6_18_18, B[6] * B[18], a[18]);
    }
  }
  template <typename T>
  static __device__ __forceinline__ void tangent(const T* B, const T* Bd, const T* d3, const T* d3d, T* Dd) {
    Dd[0] = fma(Bd[0], d3[0], B[0] * d3d[0]);
    Dd[1] = fma(Bd[0], d3[1], B[0] * d3d[1]);
    Dd[2] = fma(Bd[0], d3[2], B[0] * d3d[2]);
    Dd[3] = (Bd[1] * B[1] * B[4] + B[1] * Bd[1] * B[4] + B[1] * B[1] * Bd[4]) + T(2) * (Bd[1] * B[2] * B[7] + B[1] * Bd[2] * B[7] + B[1] * B[2] * Bd[7]) + T(2) * (Bd[1] * B[3] * B[8] + B[1] * Bd[3] * B[8] + B[1] * B[3] * Bd[8]) + (Bd[2] * B[2] * B[5] + B[2] * Bd[2] * B[5] + B[2] * B[2] * Bd[5]) + T(2) * (Bd[2] * B[3] * B[9] + B[2] * Bd[3] * B[9] + B[2] * B[3] * Bd[9]) + (Bd[3] * B[3] * B[6] + B[3] * Bd[3] * B[6] + B[3] * B[3] * Bd[6]);
    Dd[4] = fma(Bd[0], d3[3], B[0] * d3d[3]);
    Dd[5] = (Bd[1] * B[4] * B[10] + B[1] * Bd[4] * B[10] + B[1] * B[4] * Bd[10]) + (Bd[2] * B[4] * B[13] + B[2] * Bd[4] * B[13] + B[2] * B[4] * Bd[13]) + (Bd[3] * B[4] * B[14] + B[3] * Bd[4] * B[14] + B[3] * B[4] * Bd[14]) + (Bd[1] * B[5] * B[15] + B[1] * Bd[5] * B[15] + B[1] * B[5] * Bd[15]) + (Bd[2] * B[5] * B[11] + B[2] * Bd[5] * B[11] + B[2] * B[5] * Bd[11]) + (Bd[3] * B[5] * B[16] + B[3] * Bd[5] * B[16] + B[3] * B[5] * Bd[16]) + (Bd[1] * B[6] * B[17] + B[1] * Bd[6] * B[17] + B[1] * B[6] * Bd[17]) + (Bd[2] * B[6] * B[18] + B[2] * Bd[6] * B[18] + B[2] * B[6] * Bd[18]) + (Bd[3] * B[6] * B[12] + B[3] * Bd[6] * B[12] + B[3] * B[6] * Bd[12]) + T(2) * (Bd[1] * B[7] * B[13] + B[1] * Bd[7] * B[13] + B[1] * B[7] * Bd[13]) + T(2) * (Bd[2] * B[7] * B[15] + B[2] * Bd[7] * B[15] + B[2] * B[7] * Bd[15]) + T(2) * (Bd[3] * B[7] * B[19] + B[3] * Bd[7] * B[19] + B[3] * B[7] * Bd[19]) + T(2) * (Bd[1] * B[8] * B[14] + B[1] * Bd[8] * B[14] + B[1] * B[8] * Bd[14]) + T(2) * (Bd[2] * B[8] * B[19] + B[2] * Bd[8] * B[19] + B[2] * B[8] * Bd[19]) + T(2) * (Bd[3] * B[8] * B[17] + B[3] * Bd[8] * B[17] + B[3] * B[8] * Bd[17]) + T(2) * (Bd[1] * B[9] * B[19] + B[1] * Bd[9] * B[19] + B[1] * B[9] * Bd[19]) + T(2) * (Bd[2] * B[9] * B[16] + B[2] * Bd[9] * B[16] + B[2] * B[9] * Bd[16]) + T(2) * (Bd[3] * B[9] * B[18] + B[3] * Bd[9] * B[18] + B[3] * B[9] * Bd[18]);
    Dd[6] = (Bd[4] * B[4] * B[4] + B[4] * Bd[4] * B[4] + B[4] * B[4] * Bd[4]) + T(3) * (Bd[4] * B[7] * B[7] + B[4] * Bd[7] * B[7] + B[4] * B[7] * Bd[7]) + T(3) * (Bd[4] * B[8] * B[8] + B[4] * Bd[8] * B[8] + B[4] * B[8] * Bd[8]) + T(3) * (Bd[5] * B[7] * B[7] + B[5] * Bd[7] * B[7] + B[5] * B[7] * Bd[7]) + T(6) * (Bd[7] * B[8] * B[9] + B[7] * Bd[8] * B[9] + B[7] * B[8] * Bd[9]) + T(3) * (Bd[6] * B[8] * B[8] + B[6] * Bd[8] * B[8] + B[6] * B[8] * Bd[8]) + (Bd[5] * B[5] * B[5] + B[5] * Bd[5] * B[5] + B[5] * B[5] * Bd[5]) + T(3) * (Bd[5] * B[9] * B[9] + B[5] * Bd[9] * B[9] + B[5] * B[9] * Bd[9]) + T(3) * (Bd[6] * B[9] * B[9] + B[6] * Bd[9] * B[9] + B[6] * B[9] * Bd[9]) + (Bd[6] * B[6] * B[6] + B[6] * Bd[6] * B[6] + B[6] * B[6] * Bd[6]);
    Dd[7] = fma(Bd[0], d3[4], B[0] * d3d[4]);
    Dd[8] = (Bd[1] * B[10] * B[20] + B[1] * Bd[10] * B[20] + B[1] * B[10] * Bd[20]) + (Bd[2] * B[10] * B[23] + B[2] * Bd[10] * B[23] + B[2] * B[10] * Bd[23]) + (Bd[3] * B[10] * B[24] + B[3] * Bd[10] * B[24] + B[3] * B[10] * Bd[24]) + (Bd[1] * B[11] * B[25] + B[1] * Bd[11] * B[25] + B[1] * B[11] * Bd[25]) + (Bd[2] * B[11] * B[21] + B[2] * Bd[11] * B[21] + B[2] * B[11] * Bd[21]) + (Bd[3] * B[11] * B[26] + B[3] * Bd[11] * B[26] + B[3] * B[11] * Bd[26]) + (Bd[1] * B[12] * B[27] + B[1] * Bd[12] * B[27] + B[1] * B[12] * Bd[27]) + (Bd[2] * B[12] * B[28] + B[2] * Bd[12] * B[28] + B[2] * B[12] * Bd[28]) + (Bd[3] * B[12] * B[22] + B[3] * Bd[12] * B[22] + B[3] * B[12] * Bd[22]) + T(3) * (Bd[1] * B[13] * B[23] + B[1] * Bd[13] * B[23] + B[1] * B[13] * Bd[23]) + T(3) * (Bd[2] * B[13] * B[29] + B[2] * Bd[13] * B[29] + B[2] * B[13] * Bd[29]) + T(3) * (Bd[3] * B[13] * B[32] + B[3] * Bd[13] * B[32] + B[3] * B[13] * Bd[32]) + T(3) * (Bd[1] * B[14] * B[24] + B[1] * Bd[14] * B[24] + B[1] * B[14] * Bd[24]) + T(3) * (Bd[2] * B[14] * B[32] + B[2] * Bd[14] * B[32] + B[2] * B[14] * Bd[32]) + T(3) * (Bd[3] * B[14] * B[30] + B[3] * Bd[14] * B[30] + B[3] * B[14] * Bd[30]) + T(3) * (Bd[1] * B[15] * B[29] + B[1] * Bd[15] * B[29] + B[1] * B[15] * Bd[29]) + T(3) * (Bd[2] * B[15] * B[25] + B[2] * Bd[15] * B[25] + B[2] * B[15] * Bd[25]) + T(3) * (Bd[3] * B[15] * B[33] + B[3] * Bd[15] * B[33] + B[3] * B[15] * Bd[33]) + T(3) * (Bd[1] * B[16] * B[33] + B[1] * Bd[16] * B[33] + B[1] * B[16] * Bd[33]) + T(3) * (Bd[2] * B[16] * B[26] + B[2] * Bd[16] * B[26] + B[2] * B[16] * Bd[26]) + T(3) * (Bd[3] * B[16] * B[31] + B[3] * Bd[16] * B[31] + B[3] * B[16] * Bd[31]) + T(3) * (Bd[1] * B[17] * B[30] + B[1] * Bd[17] * B[30] + B[1] * B[17] * Bd[30]) + T(3) * (Bd[2] * B[17] * B[34] + B[2] * Bd[17] * B[34] + B[2] * B[17] * Bd[34]) + T(3) * (Bd[3] * B[17] * B[27] + B[3] * Bd[17] * B[27] + B[3] * B[17] * Bd[27]) + T(3) * (Bd[1] * B[18] * B[34] + B[1] * Bd[18] * B[34] + B[1] * B[18] * Bd[34]) + T(3) * (Bd[2] * B[18] * B[31] + B[2] * Bd[18] * B[31] + B[2] * B[18] * Bd[31]) + T(3) * (Bd[3] * B[18] * B[28] + B[3] * Bd[18] * B[28] + B[3] * B[18] * Bd[28]) + T(6) * (Bd[1] * B[19] * B[32] + B[1] * Bd[19] * B[32] + B[1] * B[19] * Bd[32]) + T(6) * (Bd[2] * B[19] * B[33] + B[2] * Bd[19] * B[33] + B[2] * B[19] * Bd[33]) + T(6) * (Bd[3] * B[19] * B[34] + B[3] * Bd[19] * B[34] + B[3] * B[19] * Bd[34]);
    Dd[9] = (Bd[4] * B[4] * B[20] + B[4] * Bd[4] * B[20] + B[4] * B[4] * Bd[20]) + T(2) * (Bd[4] * B[5] * B[29] + B[4] * Bd[5] * B[29] + B[4] * B[5] * Bd[29]) + T(2) * (Bd[4] * B[6] * B[30] + B[4] * Bd[6] * B[30] + B[4] * B[6] * Bd[30]) + T(4) * (Bd[4] * B[7] * B[23] + B[4] * Bd[7] * B[23] + B[4] * B[7] * Bd[23]) + T(4) * (Bd[4] * B[8] * B[24] + B[4] * Bd[8] * B[24] + B[4] * B[8] * Bd[24]) + T(4) * (Bd[4] * B[9] * B[32] + B[4] * Bd[9] * B[32] + B[4] * B[9] * Bd[32]) + (Bd[5] * B[5] * B[21] + B[5] * Bd[5] * B[21] + B[5] * B[5] * Bd[21]) + T(2) * (Bd[5] * B[6] * B[31] + B[5] * Bd[6] * B[31] + B[5] * B[6] * Bd[31]) + T(4) * (Bd[5] * B[7] * B[25] + B[5] * Bd[7] * B[25] + B[5] * B[7] * Bd[25]) + T(4) * (Bd[5] * B[8] * B[33] + B[5] * Bd[8] * B[33] + B[5] * B[8] * Bd[33]) + T(4) * (Bd[5] * B[9] * B[26] + B[5] * Bd[9] * B[26] + B[5] * B[9] * Bd[26]) + (Bd[6] * B[6] * B[22] + B[6] * Bd[6] * B[22] + B[6] * B[6] * Bd[22]) + T(4) * (Bd[6] * B[7] * B[34] + B[6] * Bd[7] * B[34] + B[6] * B[7] * Bd[34]) + T(4) * (Bd[6] * B[8] * B[27] + B[6] * Bd[8] * B[27] + B[6] * B[8] * Bd[27]) + T(4) * (Bd[6] * B[9] * B[28] + B[6] * Bd[9] * B[28] + B[6] * B[9] * Bd[28]) + T(4) * (Bd[7] * B[7] * B[29] + B[7] * Bd[7] * B[29] + B[7] * B[7] * Bd[29]) + T(8) * (Bd[7] * B[8] * B[32] + B[7] * Bd[8] * B[32] + B[7] * B[8] * Bd[32]) + T(8) * (Bd[7] * B[9] * B[33] + B[7] * Bd[9] * B[33] + B[7] * B[9] * Bd[33]) + T(4) * (Bd[8] * B[8] * B[30] + B[8] * Bd[8] * B[30] + B[8] * B[8] * Bd[30]) + T(8) * (Bd[8] * B[9] * B[34] + B[8] * Bd[9] * B[34] + B[8] * B[9] * Bd[34]) + T(4) * (Bd[9] * B[9] * B[31] + B[9] * Bd[9] * B[31] + B[9] * B[9] * Bd[31]);
    Dd[10] = (Bd[4] * B[10] * B[10] + B[4] * Bd[10] * B[10] + B[4] * B[10] * Bd[10]) + T(2) * (Bd[7] * B[10] * B[13] + B[7] * Bd[10] * B[13] + B[7] * B[10] * Bd[13]) + T(2) * (Bd[8] * B[10] * B[14] + B[8] * Bd[10] * B[14] + B[8] * B[10] * Bd[14]) + (Bd[5] * B[13] * B[13] + B[5] * Bd[13] * B[13] + B[5] * B[13] * Bd[13]) + T(2) * (Bd[9] * B[13] * B[14] + B[9] * Bd[13] * B[14] + B[9] * B[13] * Bd[14]) + (Bd[6] * B[14] * B[14] + B[6] * Bd[14] * B[14] + B[6] * B[14] * Bd[14]) + (Bd[4] * B[15] * B[15] + B[4] * Bd[15] * B[15] + B[4] * B[15] * Bd[15]) + T(2) * (Bd[7] * B[11] * B[15] + B[7] * Bd[11] * B[15] + B[7] * B[11] * Bd[15]) + T(2) * (Bd[8] * B[15] * B[16] + B[8] * Bd[15] * B[16] + B[8] * B[15] * Bd[16]) + (Bd[5] * B[11] * B[11] + B[5] * Bd[11] * B[11] + B[5] * B[11] * Bd[11]) + T(2) * (Bd[9] * B[11] * B[16] + B[9] * Bd[11] * B[16] + B[9] * B[11] * Bd[16]) + (Bd[6] * B[16] * B[16] + B[6] * Bd[16] * B[16] + B[6] * B[16] * Bd[16]) + (Bd[4] * B[17] * B[17] + B[4] * Bd[17] * B[17] + B[4] * B[17] * Bd[17]) + T(2) * (Bd[7] * B[17] * B[18] + B[7] * Bd[17] * B[18] + B[7] * B[17] * Bd[18]) + T(2) * (Bd[8] * B[12] * B[17] + B[8] * Bd[12] * B[17] + B[8] * B[12] * Bd[17]) + (Bd[5] * B[18] * B[18] + B[5] * Bd[18] * B[18] + B[5] * B[18] * Bd[18]) + T(2) * (Bd[9] * B[12] * B[18] + B[9] * Bd[12] * B[18] + B[9] * B[12] * Bd[18]) + (Bd[6] * B[12] * B[12] + B[6] * Bd[12] * B[12] + B[6] * B[12] * Bd[12]) + T(2) * (Bd[4] * B[13] * B[13] + B[4] * Bd[13] * B[13] + B[4] * B[13] * Bd[13]) + T(4) * (Bd[7] * B[13] * B[15] + B[7] * Bd[13] * B[15] + B[7] * B[13] * Bd[15]) + T(4) * (Bd[8] * B[13] * B[19] + B[8] * Bd[13] * B[19] + B[8] * B[13] * Bd[19]) + T(2) * (Bd[5] * B[15] * B[15] + B[5] * Bd[15] * B[15] + B[5] * B[15] * Bd[15]) + T(4) * (Bd[9] * B[15] * B[19] + B[9] * Bd[15] * B[19] + B[9] * B[15] * Bd[19]) + T(2) * (Bd[6] * B[19] * B[19] + B[6] * Bd[19] * B[19] + B[6] * B[19] * Bd[19]) + T(2) * (Bd[4] * B[14] * B[14] + B[4] * Bd[14] * B[14] + B[4] * B[14] * Bd[14]) + T(4) * (Bd[7] * B[14] * B[19] + B[7] * Bd[14] * B[19] + B[7] * B[14] * Bd[19]) + T(4) * (Bd[8] * B[14] * B[17] + B[8] * Bd[14] * B[17] + B[8] * B[14] * Bd[17]) + T(2) * (Bd[5] * B[19] * B[19] + B[5] * Bd[19] * B[19] + B[5] * B[19] * Bd[19]) + T(4) * (Bd[9] * B[17] * B[19] + B[9] * Bd[17] * B[19] + B[9] * B[17] * Bd[19]) + T(2) * (Bd[6] * B[17] * B[17] + B[6] * Bd[17] * B[17] + B[6] * B[17] * Bd[17]) + T(2) * (Bd[4] * B[19] * B[19] + B[4] * Bd[19] * B[19] + B[4] * B[19] * Bd[19]) + T(4) * (Bd[7] * B[16] * B[19] + B[7] * Bd[16] * B[19] + B[7] * B[16] * Bd[19]) + T(4) * (Bd[8] * B[18] * B[19] + B[8] * Bd[18] * B[19] + B[8] * B[18] * Bd[19]) + T(2) * (Bd[5] * B[16] * B[16] + B[5] * Bd[16] * B[16] + B[5] * B[16] * Bd[16]) + T(4) * (Bd[9] * B[16] * B[18] + B[9] * Bd[16] * B[18] + B[9] * B[16] * Bd[18]) + T(2) * (Bd[6] * B[18] * B[18] + B[6] * Bd[18] * B[18] + B[6] * B[18] * Bd[18]);
  }
  static constexpr int NTERMS = 121;
};
