// Small complex type for device and host code (double and float).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#define LMF_HD __host__ __device__ __forceinline__

template <typename T>
struct cx {
    T x, y;
};
using cd = cx<double>;
using cf = cx<float>;

template <typename T> LMF_HD cx<T> mk(T a, T b) { return cx<T>{a, b}; }
LMF_HD cd mkd(double a, double b = 0.0) { return cd{a, b}; }

template <typename T> LMF_HD cx<T> operator+(cx<T> a, cx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T> LMF_HD cx<T> operator-(cx<T> a, cx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T> LMF_HD cx<T> operator-(cx<T> a) { return {-a.x, -a.y}; }
template <typename T> LMF_HD cx<T> operator*(cx<T> a, cx<T> b)
{
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> LMF_HD cx<T> operator*(T s, cx<T> a) { return {s * a.x, s * a.y}; }
template <typename T> LMF_HD cx<T> operator*(cx<T> a, T s) { return {s * a.x, s * a.y}; }
template <typename T> LMF_HD cx<T> &operator+=(cx<T> &a, cx<T> b) { a.x += b.x; a.y += b.y; return a; }
template <typename T> LMF_HD cx<T> &operator-=(cx<T> &a, cx<T> b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename T> LMF_HD cx<T> conj(cx<T> a) { return {a.x, -a.y}; }
template <typename T> LMF_HD cx<T> mul_i(cx<T> a) { return {-a.y, a.x}; }      // i*a
template <typename T> LMF_HD cx<T> mul_mi(cx<T> a) { return {a.y, -a.x}; }     // -i*a
template <typename T> LMF_HD T abs2(cx<T> a) { return a.x * a.x + a.y * a.y; }
LMF_HD double cabsd(cd a) { return hypot(a.x, a.y); }

// Smith's division, robust against overflow of |b|^2
template <typename T> LMF_HD cx<T> operator/(cx<T> a, cx<T> b)
{
    if (fabs(b.x) >= fabs(b.y)) {
        T r = b.y / b.x, den = b.x + b.y * r;
        return {(a.x + a.y * r) / den, (a.y - a.x * r) / den};
    } else {
        T r = b.x / b.y, den = b.x * r + b.y;
        return {(a.x * r + a.y) / den, (a.y * r - a.x) / den};
    }
}
template <typename T> LMF_HD cx<T> operator/(cx<T> a, T s) { return {a.x / s, a.y / s}; }
template <typename T> LMF_HD cx<T> inv(cx<T> b) { return cx<T>{T(1), T(0)} / b; }

// e^z
LMF_HD cd cexpd(cd z)
{
    double e = exp(z.x), s, c;
    sincos(z.y, &s, &c);
    return {e * c, e * s};
}

// principal square root (branch cut on the negative real axis, Re >= 0)
LMF_HD cd csqrtd(cd z)
{
    double r = hypot(z.x, z.y);
    if (r == 0.0) return {0.0, 0.0};
    if (z.x >= 0.0) {
        double t = sqrt(0.5 * (r + z.x));
        return {t, z.y / (2.0 * t)};
    }
    double t = sqrt(0.5 * (r - z.x));
    return {fabs(z.y) / (2.0 * t), copysign(t, z.y)};
}

// log z, principal
LMF_HD cd clogd(cd z) { return {log(hypot(z.x, z.y)), atan2(z.y, z.x)}; }

// vertical wavenumber sqrt(k^2 - kr^2) on the sheet Im >= 0
LMF_HD cd kz_of(cd k, cd kr)
{
    cd s = csqrtd(k * k - kr * kr);
    if (s.y < 0.0) s = -s;
    return s;
}

// i^n for integer n
template <typename T> LMF_HD cx<T> ipow(int n)
{
    switch (n & 3) {
    case 0: return {T(1), T(0)};
    case 1: return {T(0), T(1)};
    case 2: return {T(-1), T(0)};
    default: return {T(0), T(-1)};
    }
}
