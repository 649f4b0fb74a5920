// Values of one or two cells for the per-cell arithmetic of the step.
//
// The tile sweep can give each thread two horizontally adjacent cells; their
// arithmetic is then written once on a pair type whose operators are the
// sm_100-family packed FP32 instructions (two lanes per instruction, each
// lane rounded exactly like the scalar operation).  V = float is the one-cell
// form; V = f2 the two-cell form; VI = int / i2 their fixed-point companions.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

struct f2 {
    float x, y;
    __device__ __forceinline__ f2() {}
    __device__ __forceinline__ f2(float a, float b) : x(a), y(b) {}
    __device__ __forceinline__ explicit f2(float s) : x(s), y(s) {}
};

struct i2 {
    int x, y;
};

__device__ __forceinline__ float2 as_f2(f2 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ f2 from_f2(float2 a) { return f2(a.x, a.y); }

__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return from_f2(__fadd2_rn(as_f2(a), as_f2(b))); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return from_f2(__fmul2_rn(as_f2(a), as_f2(b))); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
    f2 d;
    asm("{.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ f2 operator-(f2 a) { return f2(-a.x, -a.y); }
__device__ __forceinline__ f2 operator+(f2 a, float s) { return a + f2(s); }
__device__ __forceinline__ f2 operator+(float s, f2 a) { return f2(s) + a; }
__device__ __forceinline__ f2 operator-(f2 a, float s) { return a - f2(s); }
__device__ __forceinline__ f2 operator-(float s, f2 a) { return f2(s) - a; }
__device__ __forceinline__ f2 operator*(f2 a, float s) { return a * f2(s); }
__device__ __forceinline__ f2 operator*(float s, f2 a) { return f2(s) * a; }
__device__ __forceinline__ f2& operator+=(f2& a, f2 b) { return a = a + b; }
__device__ __forceinline__ f2& operator-=(f2& a, f2 b) { return a = a - b; }

// a * b + c, fused (one rounding), for both forms.
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ f2 vfma(f2 a, f2 b, f2 c) {
    return from_f2(__ffma2_rn(as_f2(a), as_f2(b), as_f2(c)));
}
__device__ __forceinline__ f2 vfma(float a, f2 b, f2 c) { return vfma(f2(a), b, c); }
__device__ __forceinline__ f2 vfma(f2 a, float b, f2 c) { return vfma(a, f2(b), c); }

// Per-lane helpers.
template <class V> struct Lanes;
template <> struct Lanes<float> {
    static constexpr int n = 1;
    using I = int;
};
template <> struct Lanes<f2> {
    static constexpr int n = 2;
    using I = i2;
};

__device__ __forceinline__ float lane(float v, int) { return v; }
__device__ __forceinline__ float lane(f2 v, int k) { return k ? v.y : v.x; }
__device__ __forceinline__ int lane(int v, int) { return v; }
__device__ __forceinline__ int lane(i2 v, int k) { return k ? v.y : v.x; }
__device__ __forceinline__ void set_lane(float& v, int, float s) { v = s; }
__device__ __forceinline__ void set_lane(f2& v, int k, float s) {
    if (k) v.y = s;
    else v.x = s;
}
__device__ __forceinline__ void set_lane(int& v, int, int s) { v = s; }
__device__ __forceinline__ void set_lane(i2& v, int k, int s) {
    if (k) v.y = s;
    else v.x = s;
}

template <class V> __device__ __forceinline__ V vsplat(float s);
template <> __device__ __forceinline__ float vsplat<float>(float s) { return s; }
template <> __device__ __forceinline__ f2 vsplat<f2>(float s) { return f2(s); }

// Integer differences and the float value of fixed-point numbers.
__device__ __forceinline__ int isub(int a, int b) { return a - b; }
__device__ __forceinline__ i2 isub(i2 a, i2 b) { return i2{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ i2 isub(int a, i2 b) { return i2{a - b.x, a - b.y}; }
__device__ __forceinline__ i2 isub(i2 a, int b) { return i2{a.x - b, a.y - b}; }
__device__ __forceinline__ float i2f(int a) { return (float)a; }
__device__ __forceinline__ f2 i2f(i2 a) { return f2((float)a.x, (float)a.y); }

// Apply a scalar function to every lane.
template <class F> __device__ __forceinline__ float vmap(float v, F f) { return f(v); }
template <class F> __device__ __forceinline__ f2 vmap(f2 v, F f) { return f2(f(v.x), f(v.y)); }

}  // namespace lbm
