// Roles of the columns pushed through each of the five M2L tables of the
// helical form (shared by the FP32/FP64 SIMT kernel and the tensor-core kernel).
#pragma once

namespace lmf {

// Column roles per table t: (input helical v, signed kappa, coefficient,
// output helical v) for
//   A' = 1/2 T0[s1] a - 1/2 T2[s3] b + T1[s2] c
//   B' = 1/2 T0[s1] b - 1/2 T-2[s3] a + T-1[s2] c
//   C' = T0[s5] c + 1/2 T-1[s4] a + 1/2 T1[s4] b
struct ColSpec {
    int vin, kap;
    double coef;
    int vout, pad;
};
static __constant__ ColSpec c_cols[5][2] = {
    {{0, 0, 0.5, 0, 0}, {1, 0, 0.5, 1, 0}},     // (s1, 0)
    {{2, 0, 1.0, 2, 0}, {2, 0, 1.0, 2, 0}},     // (s5, 0)  (one column)
    {{2, 1, 1.0, 0, 0}, {2, -1, 1.0, 1, 0}},    // (s2, 1)
    {{1, 1, 0.5, 2, 0}, {0, -1, 0.5, 2, 0}},    // (s4, 1)
    {{1, 2, -0.5, 0, 0}, {0, -2, -0.5, 1, 0}},  // (s3, 2)
};

}  // namespace lmf
