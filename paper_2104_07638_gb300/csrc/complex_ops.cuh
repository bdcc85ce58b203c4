// Complex (double2: re, im) arithmetic shared by the Keldysh kernels.
#pragma once

#include <cuda_runtime.h>

#include "apm_internal.cuh"

namespace apm {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// c - a*b
__device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 c) {
    return make_double2(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
// c + a*b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cneg_if(double2 a, bool neg) {
    return neg ? make_double2(-a.x, -a.y) : a;
}
// 1/p; flags a zero or non-finite pivot (|p|^2 == 0, inf or NaN), tested on
// the bits so that no FP64 compare is issued
__device__ __forceinline__ double2 crcp(double2 p, int &bad) {
    const double d = fma(p.x, p.x, p.y * p.y);
    const long long bits = __double_as_longlong(d);
    if (bits == 0 || ((bits >> 52) & 0x7ff) == 0x7ff) bad = 1;
    const double r = rcp_nr(d);
    return make_double2(p.x * r, -p.y * r);
}
__device__ __forceinline__ double2 warp_csum(double2 v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

}  // namespace apm
