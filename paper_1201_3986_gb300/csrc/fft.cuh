// Small complex FFT building blocks shared by the on-chip 2D FFT (fused2d.cuh)
// and the 3D FFT over global scratch (fast3d.cu): complex type per real
// type, complex product, and in-register DFTs of radix 2, 3, 4, 6 and 8.
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
    } else if constexpr (R == 6) {
        // X[k] = E[k] + w^k O[k], X[k+3] = E[k] - w^k O[k] (k < 3) with E, O
        // the 3-point DFTs of the even and odd samples, w = exp(-+ 2 pi i / 6)
        C e[3] = {v[0], v[2], v[4]};
        C o[3] = {v[1], v[3], v[5]};
        dft_small<3, INV>(e);
        dft_small<3, INV>(o);
        const S h = S(0.8660254037844386467637231707529362);  // sqrt(3)/2
        // forward: w = 1/2 - i h, w^2 = -1/2 - i h; inverse: conjugates
        const S s1 = INV ? h : -h;
        const C o1 = {S(0.5) * o[1].x - s1 * o[1].y, S(0.5) * o[1].y + s1 * o[1].x};
        const C o2 = {-S(0.5) * o[2].x - s1 * o[2].y, -S(0.5) * o[2].y + s1 * o[2].x};
        v[0] = C{e[0].x + o[0].x, e[0].y + o[0].y};
        v[3] = C{e[0].x - o[0].x, e[0].y - o[0].y};
        v[1] = C{e[1].x + o1.x, e[1].y + o1.y};
        v[4] = C{e[1].x - o1.x, e[1].y - o1.y};
        v[2] = C{e[2].x + o2.x, e[2].y + o2.y};
        v[5] = C{e[2].x - o2.x, e[2].y - o2.y};
    } else if constexpr (R == 8) {
        // X[k] = E[k] + w^k O[k], X[k+4] = E[k] - w^k O[k] (k < 4) with E, O
        // the 4-point DFTs of the even and odd samples, w = exp(-+ 2 pi i / 8)
        C e[4] = {v[0], v[2], v[4], v[6]};
        C o[4] = {v[1], v[3], v[5], v[7]};
        dft_small<4, INV>(e);
        dft_small<4, INV>(o);
        const S r = S(0.7071067811865475244008443621048490);  // 1/sqrt(2)
        // forward: w = (1 - i) r, w^2 = -i, w^3 = (-1 - i) r; inverse: conjugates
        const C o1 = INV ? C{r * (o[1].x - o[1].y), r * (o[1].x + o[1].y)}
                         : C{r * (o[1].x + o[1].y), r * (o[1].y - o[1].x)};
        const C o2 = INV ? C{-o[2].y, o[2].x} : C{o[2].y, -o[2].x};
        const C o3 = INV ? C{-r * (o[3].x + o[3].y), r * (o[3].x - o[3].y)}
                         : C{r * (o[3].y - o[3].x), -r * (o[3].x + o[3].y)};
        v[0] = C{e[0].x + o[0].x, e[0].y + o[0].y};
        v[4] = C{e[0].x - o[0].x, e[0].y - o[0].y};
        v[1] = C{e[1].x + o1.x, e[1].y + o1.y};
        v[5] = C{e[1].x - o1.x, e[1].y - o1.y};
        v[2] = C{e[2].x + o2.x, e[2].y + o2.y};
        v[6] = C{e[2].x - o2.x, e[2].y - o2.y};
        v[3] = C{e[3].x + o3.x, e[3].y + o3.y};
        v[7] = C{e[3].x - o3.x, e[3].y - o3.y};
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

