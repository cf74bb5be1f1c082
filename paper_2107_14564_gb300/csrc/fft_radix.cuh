// Radix-R inverse DFT butterflies in registers, shared by the FFT kernels.
#pragma once

#include "common.cuh"

namespace bsp {

// ---------------------------------------------------------------- radix-R inverse DFTs
// y_k = sum_j x_j exp(+2 pi i j k / R), in registers.
template <typename C, int R> struct Dft;

template <typename C> struct Dft<C, 2> {
  static __device__ __forceinline__ void run(C* v) {
    C a = v[0], b = v[1];
    v[0] = c_add(a, b);
    v[1] = c_sub(a, b);
  }
};

template <typename C> struct Dft<C, 3> {
  static __device__ __forceinline__ void run(C* v) {
    using R = decltype(C::x);
    const R h = R(0.86602540378443864676);  // sqrt(3)/2
    C s = c_add(v[1], v[2]);
    C d = c_sub(v[1], v[2]);
    C m = c_make<C>(v[0].x - R(0.5) * s.x, v[0].y - R(0.5) * s.y);
    C id = c_make<C>(-h * d.y, h * d.x);  // i * (sqrt(3)/2) * d
    v[0] = c_add(v[0], s);
    v[1] = c_add(m, id);
    v[2] = c_sub(m, id);
  }
};

template <typename C> struct Dft<C, 4> {
  static __device__ __forceinline__ void run(C* v) {
    C t0 = c_add(v[0], v[2]);
    C t1 = c_sub(v[0], v[2]);
    C t2 = c_add(v[1], v[3]);
    C t3 = c_muli(c_sub(v[1], v[3]));
    v[0] = c_add(t0, t2);
    v[1] = c_add(t1, t3);
    v[2] = c_sub(t0, t2);
    v[3] = c_sub(t1, t3);
  }
};

template <typename C> struct Dft<C, 8> {
  static __device__ __forceinline__ void run(C* v) {
    using R = decltype(C::x);
    const R c = R(0.70710678118654752440);  // sqrt(1/2)
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    Dft<C, 4>::run(e);
    Dft<C, 4>::run(o);
    // w^k o_k with w = exp(+i pi / 4)
    C o1 = c_make<C>(c * (o[1].x - o[1].y), c * (o[1].x + o[1].y));
    C o2 = c_muli(o[2]);
    C o3 = c_make<C>(-c * (o[3].x + o[3].y), c * (o[3].x - o[3].y));
    v[0] = c_add(e[0], o[0]);
    v[4] = c_sub(e[0], o[0]);
    v[1] = c_add(e[1], o1);
    v[5] = c_sub(e[1], o1);
    v[2] = c_add(e[2], o2);
    v[6] = c_sub(e[2], o2);
    v[3] = c_add(e[3], o3);
    v[7] = c_sub(e[3], o3);
  }
};

// Radix 6 and 12 by the prime-factor (Good-Thomas) mapping, which needs no twiddles between the
// factors because they are coprime: for N = N1 N2, input n = (N2 n1 + N1 n2) mod N and output
// k = (N2 (N2^-1 mod N1) k1 + N1 (N1^-1 mod N2) k2) mod N turn the length-N DFT into N2 DFTs of
// length N1 followed by N1 DFTs of length N2.
template <typename C> struct Dft<C, 6> {  // N1 = 2, N2 = 3: n = 3 n1 + 2 n2, k = 3 k1 + 4 k2 (mod 6)
  static __device__ __forceinline__ void run(C* v) {
    C a0[2] = {v[0], v[3]}, a1[2] = {v[2], v[5]}, a2[2] = {v[4], v[1]};
    Dft<C, 2>::run(a0);
    Dft<C, 2>::run(a1);
    Dft<C, 2>::run(a2);
    C b0[3] = {a0[0], a1[0], a2[0]}, b1[3] = {a0[1], a1[1], a2[1]};
    Dft<C, 3>::run(b0);
    Dft<C, 3>::run(b1);
    v[0] = b0[0]; v[4] = b0[1]; v[2] = b0[2];
    v[3] = b1[0]; v[1] = b1[1]; v[5] = b1[2];
  }
};

template <typename C> struct Dft<C, 12> {  // N1 = 4, N2 = 3: n = 3 n1 + 4 n2, k = 9 k1 + 4 k2 (mod 12)
  static __device__ __forceinline__ void run(C* v) {
    C a0[4] = {v[0], v[3], v[6], v[9]}, a1[4] = {v[4], v[7], v[10], v[1]}, a2[4] = {v[8], v[11], v[2], v[5]};
    Dft<C, 4>::run(a0);
    Dft<C, 4>::run(a1);
    Dft<C, 4>::run(a2);
    C b[4][3];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      b[k1][0] = a0[k1];
      b[k1][1] = a1[k1];
      b[k1][2] = a2[k1];
      Dft<C, 3>::run(b[k1]);
    }
    // k = 9 k1 + 4 k2 (mod 12)
    v[0] = b[0][0]; v[4] = b[0][1]; v[8] = b[0][2];
    v[9] = b[1][0]; v[1] = b[1][1]; v[5] = b[1][2];
    v[6] = b[2][0]; v[10] = b[2][1]; v[2] = b[2][2];
    v[3] = b[3][0]; v[7] = b[3][1]; v[11] = b[3][2];
  }
};

}  // namespace bsp
