// mb_df.cuh -- float-float ("df") numbers: an unevaluated sum hi + lo of two
// FP32 values with |lo| <= ulp(hi)/2, about 48 significant bits, kept in a
// float2 (x = hi, y = lo).  The solver stores every vector that carries large
// near-null components (preconditioned directions, smoother and coarse
// iterates, Krylov solutions) this way, so that differences of neighbouring
// entries keep their small structure while all arithmetic stays on the FP32
// pipe (GB300's FP64 rate is a small fraction of its FP32 rate).
// Error-free transformations: TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and the
// FMA-based TwoProduct; renormalisation by Fast2Sum (Dekker 1971).  They rely
// on IEEE round-to-nearest FP32 without reassociation (no fast-math).
#pragma once
#include <cuda_runtime.h>

namespace mb {

__host__ __device__ inline float2 df_from_double(double v) {
    float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}
__host__ __device__ inline double df_to_double(float2 a) { return (double)a.x + (double)a.y; }
// nearest FP32 value
__device__ inline float df_val(float2 a) { return a.x + a.y; }
// a - b rounded to FP32; exact hi difference when the entries are close
// (Sterbenz), so the result is accurate relative to the difference itself
__device__ inline float df_diff(float2 a, float2 b) { return (a.x - b.x) + (a.y - b.y); }

__device__ inline float2 df_fast2sum(float s, float e) {
    float h = s + e;
    return make_float2(h, e - (h - s));
}
// a + b for an FP32 b
__device__ inline float2 df_add_f(float2 a, float b) {
    float s = a.x + b;
    float bb = s - a.x;
    float e = (a.x - (s - bb)) + (b - bb);
    return df_fast2sum(s, e + a.y);
}
// a + b
__device__ inline float2 df_add(float2 a, float2 b) {
    float s = a.x + b.x;
    float bb = s - a.x;
    float e = (a.x - (s - bb)) + (b.x - bb);
    return df_fast2sum(s, e + (a.y + b.y));
}
// a * b
__device__ inline float2 df_mul(float2 a, float2 b) {
    float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
    return df_fast2sum(p, e);
}

}  // namespace mb
