// SpMV kernel template (shared by the solver drivers).
#pragma once

#include "common.cuh"

template <class T> struct SpmvOps;
template <> struct SpmvOps<double2> {
    __device__ static double2 zero() { return make_double2(0.0, 0.0); }
    __device__ static double2 madd(double2 a, double2 b, double2 c) {
        return make_double2(c.x + a.x * b.x - a.y * b.y, c.y + a.x * b.y + a.y * b.x);
    }
    __device__ static double2 shfl_down(double2 v, int o, unsigned mask) {
        return make_double2(__shfl_down_sync(mask, v.x, o), __shfl_down_sync(mask, v.y, o));
    }
};
template <> struct SpmvOps<float2> {
    __device__ static float2 zero() { return make_float2(0.f, 0.f); }
    __device__ static float2 madd(float2 a, float2 b, float2 c) {
        return make_float2(c.x + a.x * b.x - a.y * b.y, c.y + a.x * b.y + a.y * b.x);
    }
    __device__ static float2 shfl_down(float2 v, int o, unsigned mask) {
        return make_float2(__shfl_down_sync(mask, v.x, o), __shfl_down_sync(mask, v.y, o));
    }
};

// y[i] = sum_t A[i, col[t]] x[col[t]]; G lanes per row.  Each lane issues the
// column and value loads of its next K entries before it gathers x and
// before any arithmetic, so a row costs two dependent memory round trips
// whatever its length up to K G.  Columns and values are streamed past L1
// (read once); x is gathered through the read-only cache.  `halt` (may be
// null) lets a solver skip launches it has already queued once it has
// converged.
template <int G, int K, class V, class T>
__global__ void __launch_bounds__(256) spmv_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                   const V* __restrict__ val, int64_t n, const T* __restrict__ x,
                                                   T* __restrict__ y, const int* __restrict__ halt) {
    if (halt && *halt) return;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = gid / G;
    const int sub = threadIdx.x % G;
    T acc = SpmvOps<T>::zero();
    if (row < n) {
        const int32_t a = rp[row], b = rp[row + 1];
        for (int32_t base = a + sub; base < b; base += K * G) {
            int32_t c[K];
            V v[K];
            T xv[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int32_t t = base + k * G;
                c[k] = t < b ? __ldcs(&col[t]) : -1;
                v[k] = t < b ? __ldcs(&val[t]) : V{};
            }
#pragma unroll
            for (int k = 0; k < K; ++k) xv[k] = c[k] >= 0 ? __ldg(&x[c[k]]) : SpmvOps<T>::zero();
#pragma unroll
            for (int k = 0; k < K; ++k) acc = SpmvOps<T>::madd(v[k], xv[k], acc);
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        T other = SpmvOps<T>::shfl_down(acc, o, 0xffffffffu);
        acc.x += other.x;
        acc.y += other.y;
    }
    if (row < n && sub == 0) y[row] = acc;
}

// y = A x from the part-split copy of A (FP64): row i's real parts (value v,
// column c: adds v x_c) come first, in [rp[i], mid[i]), then its imaginary
// parts (value v of i v: adds i v x_c = (-v im x_c, v re x_c)) in
// [mid[i], rp[i + 1]).  Two uniform loops accumulate into one complex sum,
// the second with the operands swapped and one sign folded into the FMA: two
// FMAs per part against one x load, no operand selection and no combining
// step.  On GB300 a warp's FP64 instruction holds a sub-partition's FP64 pipe
// for 64 cycles whatever its active lanes, so FP64 warp instructions (the
// FMAs, the lanes that pad a step, the shuffle reduction) bound the kernel
// along with its memory parallelism: four lanes per row and two parts per
// lane in flight measured best on the chain (fewer lanes issue fewer FP64
// instructions but keep fewer loads in flight).
template <int G, int K, bool IMAG>
__device__ __forceinline__ void split_segment(const uint32_t* __restrict__ col, const double* __restrict__ val,
                                              const double2* __restrict__ x, int32_t a, int32_t b, int sub,
                                              double2& acc) {
    for (int32_t base = a + sub; base < b; base += K * G) {
        uint32_t c[K];
        double v[K];
        double2 xv[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int32_t t = base + k * G;
            c[k] = t < b ? __ldcs(&col[t]) : 0u;
            v[k] = t < b ? __ldcs(&val[t]) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) xv[k] = __ldg(&x[c[k]]);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (IMAG) {
                acc.x = fma(-v[k], xv[k].y, acc.x);
                acc.y = fma(v[k], xv[k].x, acc.y);
            } else {
                acc.x = fma(v[k], xv[k].x, acc.x);
                acc.y = fma(v[k], xv[k].y, acc.y);
            }
        }
    }
}

template <int G, int K>
__global__ void __launch_bounds__(256) spmv_split_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ mid,
                                                         const uint32_t* __restrict__ col,
                                                         const double* __restrict__ val, int64_t n,
                                                         const double2* __restrict__ x, double2* __restrict__ y,
                                                         const int* __restrict__ halt) {
    if (halt && *halt) return;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = gid / G;
    const int sub = threadIdx.x % G;
    double2 acc = make_double2(0.0, 0.0);
    if (row < n) {
        const int32_t a = rp[row], m = mid[row], b = rp[row + 1];
        split_segment<G, K, false>(col, val, x, a, m, sub, acc);
        split_segment<G, K, true>(col, val, x, m, b, sub, acc);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
    }
    if (row < n && sub == 0) y[row] = acc;
}

// Lanes per row of the part-split FP64 SpMV: four, or two for rows of at
// most four parts.
int spmv_split_group_size(int64_t n_rows, int64_t parts);

// Lanes per row for a mean row length (FP64: the FP64 pipe is the scarce unit,
// fewer lanes per row; FP32: more lanes, more loads in flight).
int spmv_group_size(int64_t n_rows, int64_t nnz, bool fp32);
void spmv_launch(const DeviceCSR& A, const double2* x, double2* y, const int* halt, cudaStream_t s);
void spmv_launch32(const DeviceCSR& A, const float2* val32, const float2* x, float2* y, const int* halt,
                   cudaStream_t s);
