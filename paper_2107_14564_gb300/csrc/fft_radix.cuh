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

}  // namespace bsp
