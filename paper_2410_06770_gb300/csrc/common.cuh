// common.cuh -- element types, multiply-accumulate and small device helpers
// shared by the xGETT kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "internal.h"

namespace gett {

// Interleaved complex values (Sec. 5: prefixes c and z).  Complex products
// are not conjugated: (a + ib)(c + id) = (ac - bd) + i(ad + bc).
struct cf {
    float re, im;
};
struct zd {
    double re, im;
};

// bfloat16 bit pattern -> float (exact: bf16 is the top half of an fp32).
__device__ __forceinline__ float bf16_bits_to_float(uint16_t b)
{
    return __uint_as_float(static_cast<uint32_t>(b) << 16);
}

// ---------------------------------------------------------------------------
// Per-type traits: In = operand storage, Acc = arithmetic type (also the
// type held in shared memory by the CUDA-core kernels), Out = C storage.
// ---------------------------------------------------------------------------
template <class In> struct Tr;

template <> struct Tr<float> {
    using Acc = float;
    using Out = float;
    static __device__ __forceinline__ Acc load(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ Acc zero() { return 0.f; }
    static __device__ __forceinline__ void mac(Acc &c, Acc a, Acc b) { c = fmaf(a, b, c); }
    static __device__ __forceinline__ Acc add(Acc a, Acc b) { return a + b; }
    static __device__ __forceinline__ Acc mul(Acc a, Acc b) { return a * b; }
    static __device__ __forceinline__ void store_add(Out *c, Acc v) { *c = *c + v; }
    static __device__ __forceinline__ Acc load_c(const Out *c) { return *c; }
    static __device__ __forceinline__ void store_c(Out *c, Acc v) { *c = v; }
};

template <> struct Tr<double> {
    using Acc = double;
    using Out = double;
    static __device__ __forceinline__ Acc load(const double *p) { return __ldg(p); }
    static __device__ __forceinline__ Acc zero() { return 0.0; }
    static __device__ __forceinline__ void mac(Acc &c, Acc a, Acc b) { c = fma(a, b, c); }
    static __device__ __forceinline__ Acc add(Acc a, Acc b) { return a + b; }
    static __device__ __forceinline__ Acc mul(Acc a, Acc b) { return a * b; }
    static __device__ __forceinline__ void store_add(Out *c, Acc v) { *c = *c + v; }
    static __device__ __forceinline__ Acc load_c(const Out *c) { return *c; }
    static __device__ __forceinline__ void store_c(Out *c, Acc v) { *c = v; }
};

template <> struct Tr<uint16_t> {  // bfloat16 operands, float arithmetic
    using Acc = float;
    using Out = float;
    static __device__ __forceinline__ Acc load(const uint16_t *p) { return bf16_bits_to_float(__ldg(p)); }
    static __device__ __forceinline__ Acc zero() { return 0.f; }
    static __device__ __forceinline__ void mac(Acc &c, Acc a, Acc b) { c = fmaf(a, b, c); }
    static __device__ __forceinline__ Acc add(Acc a, Acc b) { return a + b; }
    static __device__ __forceinline__ Acc mul(Acc a, Acc b) { return a * b; }
    static __device__ __forceinline__ void store_add(Out *c, Acc v) { *c = *c + v; }
    static __device__ __forceinline__ Acc load_c(const Out *c) { return *c; }
    static __device__ __forceinline__ void store_c(Out *c, Acc v) { *c = v; }
};

template <> struct Tr<cf> {
    using Acc = cf;
    using Out = cf;
    static __device__ __forceinline__ Acc load(const cf *p)
    {
        float2 v = __ldg(reinterpret_cast<const float2 *>(p));
        return cf{v.x, v.y};
    }
    static __device__ __forceinline__ Acc zero() { return cf{0.f, 0.f}; }
    static __device__ __forceinline__ void mac(Acc &c, Acc a, Acc b)
    {
        c.re = fmaf(a.re, b.re, c.re);
        c.re = fmaf(-a.im, b.im, c.re);
        c.im = fmaf(a.re, b.im, c.im);
        c.im = fmaf(a.im, b.re, c.im);
    }
    static __device__ __forceinline__ Acc add(Acc a, Acc b) { return cf{a.re + b.re, a.im + b.im}; }
    static __device__ __forceinline__ Acc mul(Acc a, Acc b)
    {
        return cf{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
    }
    static __device__ __forceinline__ void store_add(Out *c, Acc v)
    {
        float2 *p = reinterpret_cast<float2 *>(c);
        float2 o = *p;
        o.x += v.re;
        o.y += v.im;
        *p = o;
    }
    static __device__ __forceinline__ Acc load_c(const Out *c)
    {
        float2 o = *reinterpret_cast<const float2 *>(c);
        return cf{o.x, o.y};
    }
    static __device__ __forceinline__ void store_c(Out *c, Acc v)
    {
        *reinterpret_cast<float2 *>(c) = make_float2(v.re, v.im);
    }
};

template <> struct Tr<zd> {
    using Acc = zd;
    using Out = zd;
    static __device__ __forceinline__ Acc load(const zd *p)
    {
        double2 v = __ldg(reinterpret_cast<const double2 *>(p));
        return zd{v.x, v.y};
    }
    static __device__ __forceinline__ Acc zero() { return zd{0.0, 0.0}; }
    static __device__ __forceinline__ void mac(Acc &c, Acc a, Acc b)
    {
        c.re = fma(a.re, b.re, c.re);
        c.re = fma(-a.im, b.im, c.re);
        c.im = fma(a.re, b.im, c.im);
        c.im = fma(a.im, b.re, c.im);
    }
    static __device__ __forceinline__ Acc add(Acc a, Acc b) { return zd{a.re + b.re, a.im + b.im}; }
    static __device__ __forceinline__ Acc mul(Acc a, Acc b)
    {
        return zd{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
    }
    static __device__ __forceinline__ void store_add(Out *c, Acc v)
    {
        double2 *p = reinterpret_cast<double2 *>(c);
        double2 o = *p;
        o.x += v.re;
        o.y += v.im;
        *p = o;
    }
    static __device__ __forceinline__ Acc load_c(const Out *c)
    {
        double2 o = *reinterpret_cast<const double2 *>(c);
        return zd{o.x, o.y};
    }
    static __device__ __forceinline__ void store_c(Out *c, Acc v)
    {
        *reinterpret_cast<double2 *>(c) = make_double2(v.re, v.im);
    }
};

// ---------------------------------------------------------------------------
// Scaled epilogue: C <- alpha * v + beta * C, or C <- C + v (see Scale).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float scale_by(float v, double re, double) { return (float)re * v; }
__device__ __forceinline__ double scale_by(double v, double re, double) { return re * v; }
__device__ __forceinline__ cf scale_by(cf v, double re, double im)
{
    const float a = (float)re, b = (float)im;
    return cf{a * v.re - b * v.im, a * v.im + b * v.re};
}
__device__ __forceinline__ zd scale_by(zd v, double re, double im)
{
    return zd{re * v.re - im * v.im, re * v.im + im * v.re};
}

template <class R>
__device__ __forceinline__ void epi_store(typename R::Out *c, typename R::Acc v, const Scale &sc)
{
    if (sc.mode == SCALE_ACC) {
        R::store_add(c, v);
    } else if (sc.mode == SCALE_AX) {
        R::store_c(c, scale_by(v, sc.ar, sc.ai));
    } else {
        R::store_c(c, R::add(scale_by(v, sc.ar, sc.ai), scale_by(R::load_c(c), sc.br, sc.bi)));
    }
}

// Warp shuffles for every arithmetic type (used by the reductions).
__device__ __forceinline__ float shfl_down(float v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ double shfl_down(double v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ cf shfl_down(cf v, int d)
{
    return cf{__shfl_down_sync(0xffffffffu, v.re, d), __shfl_down_sync(0xffffffffu, v.im, d)};
}
__device__ __forceinline__ zd shfl_down(zd v, int d)
{
    return zd{__shfl_down_sync(0xffffffffu, v.re, d), __shfl_down_sync(0xffffffffu, v.im, d)};
}

// Decode a flat class index (first mode fastest) into the two increments of
// a ModeList.
__device__ __forceinline__ void decode2(const ModeList &L, int64_t idx, int64_t &o0, int64_t &o1)
{
    int64_t a = 0, b = 0;
    for (int i = 0; i < L.n; ++i) {
        int64_t e = L.ext[i];
        int64_t x = idx % e;
        idx /= e;
        a += x * L.s0[i];
        b += x * L.s1[i];
    }
    o0 = a;
    o1 = b;
}

}  // namespace gett
