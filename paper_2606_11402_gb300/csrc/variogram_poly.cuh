// Generated by variogram_poly.py (Chebyshev interpolation of the functions
// named below); do not edit.
#pragma once

namespace ggp {

// (e^a - 1 - a) / a^2: degree 6 on [0.0, 1.0], max relative error 7.5e-08 in FP32
__device__ __forceinline__ float poly_m32(float x) {
  constexpr float c[7] = {5.000000000e-01f, 1.666666269e-01f, 4.166741669e-02f, 8.328885771e-03f, 1.401372137e-03f, 1.806835935e-04f, 3.685081901e-05f};
  float h = c[6];
#pragma unroll
  for (int i = 5; i >= 0; i--) h = fmaf(h, x, c[i]);
  return h;
}

// (e^a - 1 - a - a^2/3) / a^2: degree 8 on [0.0, 2.0], max relative error 1.4e-07 in FP32
__device__ __forceinline__ float poly_m52(float x) {
  constexpr float c[9] = {1.666666716e-01f, 1.666666567e-01f, 4.166689515e-02f, 8.332177065e-03f, 1.391817001e-03f, 1.942823874e-04f, 2.817603308e-05f, 1.192743525e-06f, 6.394012075e-07f};
  float h = c[8];
#pragma unroll
  for (int i = 7; i >= 0; i--) h = fmaf(h, x, c[i]);
  return h;
}

// (1 - e^-u) / u: degree 5 on [0.0, 0.5], max relative error 5.4e-08 in FP32
__device__ __forceinline__ float poly_exp1(float x) {
  constexpr float c[6] = {1.000000000e+00f, -4.999998212e-01f, 1.666624248e-01f, -4.163007438e-02f, 8.189613931e-03f, -1.123404247e-03f};
  float h = c[5];
#pragma unroll
  for (int i = 4; i >= 0; i--) h = fmaf(h, x, c[i]);
  return h;
}

}  // namespace ggp
