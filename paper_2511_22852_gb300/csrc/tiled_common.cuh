// tiled_common.cuh -- device helpers of the cell-tiled FP32 neighbour passes (the serving form's
// and the per-event mixed form's): compensated single-precision sums, the error-free combination
// of a particle's lanes, the lanes-per-particle rule, and the packed two-wide candidate layout.
#pragma once

#include <cuda_runtime.h>

namespace sphg {

// Accumulation: each lane sums runs of kRun candidates in plain FP32 (at most kRun terms, so a
// run's sum errs by <= kRun u times the sum of its terms' magnitudes, u = 2^-24) and folds
// every run into Neumaier-compensated FP32 sums; the lanes of a particle are combined in FP32
// with error-free additions (seg_csum) and each total converted to FP64 once.
// 32 terms per run (<= 2e-6 of the run's magnitudes, within the form's 1e-5) fold half as often
// as 16 (+1.5 % serving throughput measured).
constexpr int kRun = 32;

// Neumaier-compensated single-precision sum
struct CSum {
    float hi, lo;
};
__device__ __forceinline__ void cadd(CSum &s, float x)
{
    float t = s.hi + x;
    if (fabsf(s.hi) >= fabsf(x)) s.lo += (s.hi - t) + x;
    else s.lo += (x - t) + s.hi;
    s.hi = t;
}
__device__ __forceinline__ double cval(CSum s) { return (double)s.hi + (double)s.lo; }

// The lanes of a particle combined in FP32 without loss: the pairs (hi, lo) of two lanes add as
// hi = TwoSum(hi_1, hi_2) (Knuth's error-free transformation: the rounded sum and its exact
// rounding error) with the error folded into lo = lo_1 + lo_2 + err, in a fixed tree order; the
// total lands in the particle's first lane.  (The FP64 pipe, 1/64 of the FP32 rate, is then
// needed only for the one conversion of each total.)
__device__ __forceinline__ CSum seg_csum(CSum v, int l, int L)
{
    for (int o = 1; o < L; o <<= 1) {
        const float th = __shfl_down_sync(0xFFFFFFFFu, v.hi, o);
        const float tl = __shfl_down_sync(0xFFFFFFFFu, v.lo, o);
        if ((l & (2 * o - 1)) == 0 && l + o < L) {
            const float s = v.hi + th;
            const float bb = s - v.hi;
            const float err = (v.hi - (s - bb)) + (th - bb);
            v.hi = s;
            v.lo = (v.lo + tl) + err;
        }
    }
    return v;
}

// lanes per particle: the most (up to 16) for which lw warps hold all na particles in one pass
// (floor(32 / L) particles per warp, a particle's lanes inside one warp), else 1.  It depends on
// the cell and lw alone, not on the block size, so for a given lw the summation order (and the
// results) do not change with the launch shape or the batch; lw is part of the tuned shape.
__device__ __forceinline__ int lanes_per_particle(int na, int lw)
{
    for (int L = 16; L > 1; --L)
        if (lw * (32 / L) >= na) return L;
    return 1;
}

// Candidates of a staged tile go in pairs (2k, 2k + 1), laid out so that every operand of the
// packed two-wide FP32 operations (one instruction for both candidates) loads as one register
// pair: a float4 per pair holds (a_0, a_1, b_0, b_1) for two per-candidate values a and b.
// Positions are stored negated (x_a + (-x_b) rounds exactly as x_a - x_b).  An odd tile is
// padded with a candidate kFar away (its r^2 overflows to +inf: never accepted, never in the
// shell; its terms are selected away before use, and its carried values are zero).
constexpr float kFar = 3.0e19f;

__device__ __forceinline__ void put_pair(float4 *arr, int i, float a, float b)
{
    float *p = reinterpret_cast<float *>(arr + (i >> 1));
    p[i & 1] = a;
    p[2 + (i & 1)] = b;
}
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// the cubic spline in single precision without branches, for both candidates: w(q) = (2-q)^3/4
// - max(1-q,0)^3 and dw/dq = 3 max(1-q,0)^2 - 3 (2-q)^2 / 4 on 0 <= q <= 2 take t = 2 - q,
// u = max(1 - q, 0) and their squares
__device__ __forceinline__ void spline_terms2(float2 q, float2 &t2, float2 &t, float2 &u2, float2 &u)
{
    const float2 nq = make_float2(-q.x, -q.y);
    t = __fadd2_rn(make_float2(2.0f, 2.0f), nq);
    const float2 v = __fadd2_rn(make_float2(1.0f, 1.0f), nq);
    u = make_float2(fmaxf(v.x, 0.0f), fmaxf(v.y, 0.0f));
    t2 = __fmul2_rn(t, t);
    u2 = __fmul2_rn(u, u);
}

}  // namespace sphg
