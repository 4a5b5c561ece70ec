// Small complex FFT building blocks shared by the on-chip 2D FFT (fused2d.cu)
// and the 3D FFT over global scratch (fast3d.cu): complex type per real
// type, complex product, and in-register DFTs of radix 2, 3 and 4.
#pragma once

#include <cuda_runtime.h>

template <typename T>
struct Cplx;
template <>
struct Cplx<float> {
    using type = float2;
};
template <>
struct Cplx<double> {
    using type = double2;
};

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// In-register R-point DFT, forward exp(-2 pi i q k / R) or inverse.
template <int R, bool INV, typename C>
__device__ __forceinline__ void dft_small(C (&v)[R]) {
    using S = decltype(v[0].x);
    if constexpr (R == 2) {
        const C a = v[0], b = v[1];
        v[0].x = a.x + b.x;
        v[0].y = a.y + b.y;
        v[1].x = a.x - b.x;
        v[1].y = a.y - b.y;
    } else if constexpr (R == 3) {
        const S h = S(0.8660254037844386467637231707529362);  // sqrt(3)/2
        const C t1 = {v[1].x + v[2].x, v[1].y + v[2].y};
        const C t2 = {v[1].x - v[2].x, v[1].y - v[2].y};
        const C m = {v[0].x - S(0.5) * t1.x, v[0].y - S(0.5) * t1.y};
        // forward: y1 = m - i h t2, y2 = m + i h t2 (inverse: signs swapped)
        const S sx = INV ? -h * t2.y : h * t2.y;
        const S sy = INV ? h * t2.x : -h * t2.x;
        v[0].x += t1.x;
        v[0].y += t1.y;
        v[1].x = m.x + sx;
        v[1].y = m.y + sy;
        v[2].x = m.x - sx;
        v[2].y = m.y - sy;
    } else {  // R == 4
        const C a0 = {v[0].x + v[2].x, v[0].y + v[2].y};
        const C a1 = {v[0].x - v[2].x, v[0].y - v[2].y};
        const C b0 = {v[1].x + v[3].x, v[1].y + v[3].y};
        const C b1 = {v[1].x - v[3].x, v[1].y - v[3].y};
        // forward: (-i) b1 = (b1.y, -b1.x); inverse: (+i) b1 = (-b1.y, b1.x)
        const C rb = INV ? C{-b1.y, b1.x} : C{b1.y, -b1.x};
        v[0] = C{a0.x + b0.x, a0.y + b0.y};
        v[2] = C{a0.x - b0.x, a0.y - b0.y};
        v[1] = C{a1.x + rb.x, a1.y + rb.y};
        v[3] = C{a1.x - rb.x, a1.y - rb.y};
    }
}

