// Device helpers of libgint: orbital evaluation (spline radial x real solid harmonic),
// bounded waits and the status word.
#pragma once
#include <cuda_runtime.h>

#include "gint_internal.h"

namespace gint {

// Real harmonics (no Condon-Shortley phase), per l ordered m = 0, +1, -1, +2, -2, written as
// Y_lm(r_hat) = S_lm(d) / r^l with the solid harmonics
//   S_00 = c0
//   S_1m = c1 (z, x, y)
//   S_2m = (c20 (2z^2 - x^2 - y^2), c21 xz, c21 yz, c22 (x^2 - y^2), c21 xy)
// c0 = 1/(2 sqrt(pi)), c1 = sqrt(3/(4 pi)), c20 = sqrt(5/(16 pi)), c21 = sqrt(15/(4 pi)),
// c22 = sqrt(15/(16 pi)) (orthonormal on the unit sphere).
template <typename T>
struct YC {
    static constexpr T c0 = T(0.28209479177387814347);
    static constexpr T c1 = T(0.48860251190291992159);
    static constexpr T c20 = T(0.31539156525252000603);
    static constexpr T c21 = T(1.09254843059207907054);
    static constexpr T c22 = T(0.54627421529603953527);
};

template <typename T>
__device__ __forceinline__ T dsqrt(T x);
template <>
__device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }

// spline record of radial ir at interval i (coefficients of c0 + c1 t + c2 t^2 + c3 t^3)
template <typename T>
struct Coef;
template <>
struct Coef<double> {
    double c0, c1, c2, c3;
    __device__ __forceinline__ void load(const Plan &P, int rec)
    {
        const double2 *p = reinterpret_cast<const double2 *>(P.coef64) + 2 * rec;
        double2 a = __ldg(p), b = __ldg(p + 1);
        c0 = a.x; c1 = a.y; c2 = b.x; c3 = b.y;
    }
};
template <>
struct Coef<float> {
    float c0, c1, c2, c3;
    __device__ __forceinline__ void load(const Plan &P, int rec)
    {
        float4 a = __ldg(P.coef32 + rec);
        c0 = a.x; c1 = a.y; c2 = a.z; c3 = a.w;
    }
};

template <typename T>
__device__ __forceinline__ T rcut_of(const DevSpecies &S);
template <>
__device__ __forceinline__ double rcut_of<double>(const DevSpecies &S) { return S.rcut; }
template <>
__device__ __forceinline__ float rcut_of<float>(const DevSpecies &S) { return S.rcut_f; }
template <typename T>
__device__ __forceinline__ T invdr_of(const DevSpecies &S);
template <>
__device__ __forceinline__ double invdr_of<double>(const DevSpecies &S) { return S.inv_dr; }
template <>
__device__ __forceinline__ float invdr_of<float>(const DevSpecies &S) { return S.inv_dr_f; }

// Evaluate every orbital of species `sp` at displacement d = r - centre.  emit(o, phi) is
// called for o = 0 .. norb-1 in order; with GRAD, emit(o, phi, gx, gy, gz) with the
// gradient with respect to r.  Outside the cutoff all values are 0.
template <typename T, bool GRAD, typename Emit>
__device__ __forceinline__ void eval_orbitals(const Plan &P, int sp, T dx, T dy, T dz, Emit &&emit)
{
    const DevSpecies &S = P.sp[sp];
    const T rc = rcut_of<T>(S);
    const T r2 = dx * dx + dy * dy + dz * dz;
    const int nrad = S.nrad;
    if (!(r2 < rc * rc)) {
        int o = 0;
        for (int ir = 0; ir < nrad; ++ir) {
            int nm = 2 * S.l[ir] + 1;
            for (int m = 0; m < nm; ++m, ++o) {
                if constexpr (GRAD) emit(o, T(0), T(0), T(0), T(0));
                else emit(o, T(0));
            }
        }
        return;
    }
    const T inv_dr = invdr_of<T>(S);
    const T r = dsqrt<T>(r2);
    if (r < T(1e-12)) {
        // limits at the centre: phi = f(0) c0 for l = 0, grad phi = f'(0) c1 e_m for l = 1
        int o = 0;
        for (int ir = 0; ir < nrad; ++ir) {
            Coef<T> c;
            c.load(P, S.coef_off + ir);
            int l = S.l[ir];
            if (l == 0) {
                if constexpr (GRAD) emit(o, c.c0 * YC<T>::c0, T(0), T(0), T(0));
                else emit(o, c.c0 * YC<T>::c0);
                ++o;
            } else if (l == 1) {
                T g = c.c1 * inv_dr * YC<T>::c1;
                if constexpr (GRAD) {
                    emit(o, T(0), T(0), T(0), g);
                    emit(o + 1, T(0), g, T(0), T(0));
                    emit(o + 2, T(0), T(0), g, T(0));
                } else {
                    emit(o, T(0)); emit(o + 1, T(0)); emit(o + 2, T(0));
                }
                o += 3;
            } else {
                for (int m = 0; m < 5; ++m, ++o) {
                    if constexpr (GRAD) emit(o, T(0), T(0), T(0), T(0));
                    else emit(o, T(0));
                }
            }
        }
        return;
    }
    T x = r * inv_dr;
    int i = (int)x;
    if (i > S.nint - 1) i = S.nint - 1;
    const T t = x - T(i);
    const int rec0 = S.coef_off + i * nrad;
    const T ir1 = T(1) / r;
    const T ux = dx * ir1, uy = dy * ir1, uz = dz * ir1;
    int o = 0;
    for (int ir = 0; ir < nrad; ++ir) {
        Coef<T> c;
        c.load(P, rec0 + ir);
        const T f = c.c0 + t * (c.c1 + t * (c.c2 + t * c.c3));
        const int l = S.l[ir];
        if constexpr (!GRAD) {
            if (l == 0) {
                emit(o, f * YC<T>::c0);
                o += 1;
            } else if (l == 1) {
                const T a = f * YC<T>::c1;
                emit(o, a * uz); emit(o + 1, a * ux); emit(o + 2, a * uy);
                o += 3;
            } else {
                emit(o, f * YC<T>::c20 * (T(2) * uz * uz - ux * ux - uy * uy));
                emit(o + 1, f * YC<T>::c21 * ux * uz);
                emit(o + 2, f * YC<T>::c21 * uy * uz);
                emit(o + 3, f * YC<T>::c22 * (ux * ux - uy * uy));
                emit(o + 4, f * YC<T>::c21 * ux * uy);
                o += 5;
            }
        } else {
            const T df = (c.c1 + t * (T(2) * c.c2 + T(3) * t * c.c3)) * inv_dr;
            if (l == 0) {
                const T a = df * YC<T>::c0;
                emit(o, f * YC<T>::c0, a * ux, a * uy, a * uz);
                o += 1;
            } else if (l == 1) {
                // phi = g S, g = f/r, grad = g' u S + g grad S, g' = (f' - f/r)/r
                const T g = f * ir1;
                const T gp = (df - g) * ir1;
                const T c1 = YC<T>::c1;
                const T Sz = c1 * dz, Sx = c1 * dx, Sy = c1 * dy;
                const T gc = g * c1;
                emit(o, g * Sz, gp * ux * Sz, gp * uy * Sz, gp * uz * Sz + gc);
                emit(o + 1, g * Sx, gp * ux * Sx + gc, gp * uy * Sx, gp * uz * Sx);
                emit(o + 2, g * Sy, gp * ux * Sy, gp * uy * Sy + gc, gp * uz * Sy);
                o += 3;
            } else {
                // g = f/r^2, g' = f'/r^2 - 2 f/r^3
                const T g = f * ir1 * ir1;
                const T gp = (df - T(2) * f * ir1) * ir1 * ir1;
                const T c20 = YC<T>::c20, c21 = YC<T>::c21, c22 = YC<T>::c22;
                T Sv, gxs, gys, gzs;
                Sv = c20 * (T(2) * dz * dz - dx * dx - dy * dy);
                gxs = -T(2) * c20 * dx; gys = -T(2) * c20 * dy; gzs = T(4) * c20 * dz;
                emit(o, g * Sv, gp * ux * Sv + g * gxs, gp * uy * Sv + g * gys, gp * uz * Sv + g * gzs);
                Sv = c21 * dx * dz;
                emit(o + 1, g * Sv, gp * ux * Sv + g * c21 * dz, gp * uy * Sv, gp * uz * Sv + g * c21 * dx);
                Sv = c21 * dy * dz;
                emit(o + 2, g * Sv, gp * ux * Sv, gp * uy * Sv + g * c21 * dz, gp * uz * Sv + g * c21 * dy);
                Sv = c22 * (dx * dx - dy * dy);
                emit(o + 3, g * Sv, gp * ux * Sv + T(2) * g * c22 * dx, gp * uy * Sv - T(2) * g * c22 * dy, gp * uz * Sv);
                Sv = c21 * dx * dy;
                emit(o + 4, g * Sv, gp * ux * Sv + g * c21 * dy, gp * uy * Sv + g * c21 * dx, gp * uz * Sv);
                o += 5;
            }
        }
    }
}

// Displacement of local point (a, b, c) of a batch from a slot's centre.  FP64 directly;
// FP32 as (d0_hi + off_hi) + (d0_lo + off_lo) so that the rounding error is relative to |d|
// rather than to |d0| (d0 can be ~8 bohr while |d| ~ 1 bohr dominates the integrals).
__device__ __forceinline__ void point_offset64(const Plan &P, int a, int b, int c, double *off)
{
    for (int q = 0; q < 3; ++q) off[q] = a * P.h[q] + b * P.h[3 + q] + c * P.h[6 + q];
}

__device__ __forceinline__ void split_f32(double x, float &hi, float &lo)
{
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

// One scatter of a contraction element (mu in slot a, nu in slot b) with the canonical
// rule.  `both` = the element (nu, mu) was also computed by this batch.
__device__ __forceinline__ void scatter_elem(double *H, const int *tbl, int ns, int a, int oa, int na, int b, int ob,
                                             int nbo, double val, bool both)
{
    int e = tbl[a * ns + b];
    if (e < 0) return;
    int off = e >> 1;
    bool canon = e & 1;
    if (both) {
        // self-partner blocks (a == b) keep only their upper triangle; the mirror fills the rest
        if (canon && (a != b || oa <= ob)) atomicAdd(H + off + oa * nbo + ob, val);
        return;
    }
    if (a == b) {
        atomicAdd(H + off + min(oa, ob) * na + max(oa, ob), val);
    } else if (canon) {
        atomicAdd(H + off + oa * nbo + ob, val);
    } else {
        int e2 = tbl[b * ns + a];
        atomicAdd(H + (e2 >> 1) + ob * na + oa, val);
    }
}

// FP64 -> FP32 with integer operations, round to nearest even (normal range; |x| below
// 2^-126 flushes to 0); keeps the conversion off GB300's narrow FP64 pipe.
__device__ __forceinline__ float d2f(double x)
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const uint32_t sign = (uint32_t)(b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0x7FF) return (float)x;
    const int ne = e - 1023 + 127;
    if (ne <= 0) return __uint_as_float(sign);
    if (ne >= 255) return (float)x;
    const uint64_t m = b & 0xFFFFFFFFFFFFFull;
    uint32_t mh = (uint32_t)(m >> 29);
    const uint32_t rem = (uint32_t)(m & 0x1FFFFFFFu);
    if (rem > 0x10000000u || (rem == 0x10000000u && (mh & 1u))) ++mh;
    uint32_t bits = ((uint32_t)ne << 23) + mh;   // a mantissa carry rolls into the exponent
    return __uint_as_float(sign | bits);
}

// FP32 -> FP64 in four integer operations: exact for normal numbers; zero and subnormals map
// to +-2^-127 (harmless as an addend to FP64 sums of order 1e-30 and above).
__device__ __forceinline__ double f2d_fast(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t hi = (((u & 0x7FFFFFFFu) >> 3) + 0x38000000u) | (u & 0x80000000u);
    const uint32_t lo = u << 29;
    return __hiloint2double((int)hi, (int)lo);
}

// Species descriptor for the FP32 tensor-core producers, kept in shared memory.
struct SpecSh {
    int nrad, nint, coef_off, lpack;   // lpack: 2 bits of l per radial
    float rcut2, inv_dr;
    int shape;                         // kShapeSPD / kShapeSP: radial list with a compiled evaluator
    int env_off;                       // first entry of the species' |phi| envelope (Plan::env)
};

// 2^k for -126 <= k <= 127, exactly
__device__ __forceinline__ float pow2i(int k) { return __int_as_float((127 + k) << 23); }

// Exponent k of the power-of-two scale with m 2^k < 2^14 (0 if m is 0 or not finite), kept to
// |k| <= 100 so that 2^k and 2^-k stay normal.
__device__ __forceinline__ int scale_exp(float m)
{
    if (!(m > 0.f) || !(m < 3.0e38f)) return 0;
    int e;
    frexpf(m, &e);   // m < 2^e
    return max(-100, min(100, 14 - e));
}

// A bound on |phi| of an atom image (displacement d0 = dh + dl of the batch origin from the
// image) over the points of a batch whose centre lies at bc from the origin and whose points
// lie within R of the centre: the species' envelope at the lower bound |d0 + bc| - R of their
// distance.  Written with rounded intrinsics only (no contraction), so every role of a kernel
// that evaluates it for the same image and batch gets the same bits.
__device__ __forceinline__ float phi_bound(const float *__restrict__ env, const SpecSh &S, const float *dh,
                                           const float *dl, const float *bc, float R)
{
    float d2 = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float x = __fadd_rn(__fadd_rn(dh[c], dl[c]), bc[c]);
        d2 = __fadd_rn(d2, __fmul_rn(x, x));
    }
    const float rmin = fmaxf(__fadd_rn(__fsqrt_rn(d2), -R), 0.f);
    if (!(__fmul_rn(rmin, rmin) < S.rcut2)) return 0.f;
    const int i = min((int)__fmul_rn(rmin, S.inv_dr), S.nint - 1);
    return __ldg(env + S.env_off + i);
}

// Radial lists with compiled (fully unrolled) evaluators: their radials' spline records are
// fetched together and the radials are evaluated side by side; other lists take the generic
// loop.  Order of the l values as in the species input.
template <int... Ls>
struct Shape {
    static constexpr int nrad = sizeof...(Ls);
    static constexpr int norb = ((2 * Ls + 1) + ...);
    __host__ __device__ static constexpr int l(int i)
    {
        constexpr int v[] = {Ls...};
        return v[i];
    }
};
using ShapeSPD = Shape<0, 0, 1, 1, 2>;   // 2s2p1d (13 orbitals)
using ShapeSP = Shape<0, 0, 1>;          // 2s1p (5 orbitals)
constexpr int kShapeGeneric = 0, kShapeSPD = 1, kShapeSP = 2;

__host__ __device__ constexpr int shape_of(int nrad, int lpack)
{
    return (nrad == 5 && lpack == ((0 << 0) | (0 << 2) | (1 << 4) | (1 << 6) | (2 << 8))) ? kShapeSPD
           : (nrad == 3 && lpack == ((0 << 0) | (0 << 2) | (1 << 4)))                      ? kShapeSP
                                                                                             : kShapeGeneric;
}

// phi of a compiled radial list (same conventions as eval_phi_f32), times `scale` (applied to
// the radial values, before the angular factors)
template <class SH, typename Emit>
__device__ __forceinline__ void eval_phi_shape(const SpecSh &S, const float4 *__restrict__ coef, float dx, float dy,
                                               float dz, Emit &&emit, float scale = 1.f)
{
    const float r2 = dx * dx + dy * dy + dz * dz;
    if (!(r2 < S.rcut2)) {
#pragma unroll
        for (int o = 0; o < SH::norb; ++o) emit(o, 0.f);
        return;
    }
    if (r2 < 1e-24f) {
        int o = 0;
#pragma unroll
        for (int ir = 0; ir < SH::nrad; ++ir) {
            if (SH::l(ir) == 0) emit(o, scale * __ldg(coef + S.coef_off + ir).x * YC<float>::c0);
            else
#pragma unroll
                for (int m = 0; m < 2 * SH::l(ir) + 1; ++m) emit(o + m, 0.f);
            o += 2 * SH::l(ir) + 1;
        }
        return;
    }
    float ir1 = rsqrtf(r2);
    ir1 = ir1 * (1.5f - 0.5f * r2 * ir1 * ir1);
    const float x = r2 * ir1 * S.inv_dr;
    const int i = min((int)x, S.nint - 1);
    const float t = x - (float)i;
    const float4 *cp = coef + S.coef_off + i * SH::nrad;
    float4 c[SH::nrad];
#pragma unroll
    for (int ir = 0; ir < SH::nrad; ++ir) c[ir] = __ldg(cp + ir);
    const float ux = dx * ir1, uy = dy * ir1, uz = dz * ir1;
    int o = 0;
#pragma unroll
    for (int ir = 0; ir < SH::nrad; ++ir) {
        const float f = scale * (c[ir].x + t * (c[ir].y + t * (c[ir].z + t * c[ir].w)));
        if (SH::l(ir) == 0) {
            emit(o, f * YC<float>::c0);
        } else if (SH::l(ir) == 1) {
            const float a = f * YC<float>::c1;
            emit(o, a * uz); emit(o + 1, a * ux); emit(o + 2, a * uy);
        } else {
            emit(o, f * YC<float>::c20 * (2.f * uz * uz - ux * ux - uy * uy));
            emit(o + 1, f * YC<float>::c21 * ux * uz);
            emit(o + 2, f * YC<float>::c21 * uy * uz);
            emit(o + 3, f * YC<float>::c22 * (ux * ux - uy * uy));
            emit(o + 4, f * YC<float>::c21 * ux * uy);
        }
        o += 2 * SH::l(ir) + 1;
    }
}

// FP32 orbital values of one species at displacement d (no gradient); rsqrt + one Newton
// step instead of sqrt and division.  emit(o, phi) for o = 0 .. norb-1.
// radials per species whose spline records eval_phi_f32<true> fetches all at once (the rho
// producers and the TF32 vlocal producers; the gradient evaluator and the BF16 vlocal
// producers, which hold more live values, measured faster loading them radial by radial)
constexpr int kPrefetchRad = 5;

template <bool PREFETCH = false, typename Emit>
__device__ __forceinline__ void eval_phi_f32(const SpecSh &S, const float4 *__restrict__ coef, float dx, float dy,
                                             float dz, Emit &&emit)
{
    const float r2 = dx * dx + dy * dy + dz * dz;
    const int nrad = S.nrad;
    if (!(r2 < S.rcut2)) {
        int o = 0;
        for (int ir = 0; ir < nrad; ++ir) {
            const int nm = 2 * ((S.lpack >> (2 * ir)) & 3) + 1;
            for (int m = 0; m < nm; ++m, ++o) emit(o, 0.f);
        }
        return;
    }
    if (r2 < 1e-24f) {
        int o = 0;
        for (int ir = 0; ir < nrad; ++ir) {
            const int l = (S.lpack >> (2 * ir)) & 3;
            if (l == 0) emit(o++, __ldg(coef + S.coef_off + ir).x * YC<float>::c0);
            else
                for (int m = 0; m < 2 * l + 1; ++m) emit(o++, 0.f);
        }
        return;
    }
    float ir1 = rsqrtf(r2);
    ir1 = ir1 * (1.5f - 0.5f * r2 * ir1 * ir1);
    const float r = r2 * ir1;
    const float x = r * S.inv_dr;
    int i = (int)x;
    i = min(i, S.nint - 1);
    const float t = x - (float)i;
    const float ux = dx * ir1, uy = dy * ir1, uz = dz * ir1;
    const float4 *cp = coef + S.coef_off + i * nrad;
    int o = 0;
    auto radial = [&](const float4 &c, int ir) {
        const float f = c.x + t * (c.y + t * (c.z + t * c.w));
        const int l = (S.lpack >> (2 * ir)) & 3;
        if (l == 0) {
            emit(o, f * YC<float>::c0);
            o += 1;
        } else if (l == 1) {
            const float a = f * YC<float>::c1;
            emit(o, a * uz); emit(o + 1, a * ux); emit(o + 2, a * uy);
            o += 3;
        } else {
            emit(o, f * YC<float>::c20 * (2.f * uz * uz - ux * ux - uy * uy));
            emit(o + 1, f * YC<float>::c21 * ux * uz);
            emit(o + 2, f * YC<float>::c21 * uy * uz);
            emit(o + 3, f * YC<float>::c22 * (ux * ux - uy * uy));
            emit(o + 4, f * YC<float>::c21 * ux * uy);
            o += 5;
        }
    };
    if (PREFETCH && nrad <= kPrefetchRad) {
        // all spline records of the slot are requested before the first is used, so their
        // latencies overlap instead of adding up radial by radial
        float4 c[kPrefetchRad];
#pragma unroll
        for (int ir = 0; ir < kPrefetchRad; ++ir)
            if (ir < nrad) c[ir] = __ldg(cp + ir);
#pragma unroll
        for (int ir = 0; ir < kPrefetchRad; ++ir)
            if (ir < nrad) radial(c[ir], ir);
    } else {
        for (int ir = 0; ir < nrad; ++ir) radial(__ldg(cp + ir), ir);
    }
}

// phi through the compiled evaluator of the species' radial list if it has one
template <bool PREFETCH, typename Emit>
__device__ __forceinline__ void eval_phi_any(const SpecSh &S, const float4 *__restrict__ coef, float dx, float dy,
                                             float dz, Emit &&emit)
{
    if (S.shape == kShapeSPD) eval_phi_shape<ShapeSPD>(S, coef, dx, dy, dz, emit);
    else if (S.shape == kShapeSP) eval_phi_shape<ShapeSP>(S, coef, dx, dy, dz, emit);
    else eval_phi_f32<PREFETCH>(S, coef, dx, dy, dz, emit);
}

// FP32 orbital values and gradients (with respect to r) of one species at displacement d;
// emit(o, phi, gx, gy, gz).  Same conventions as eval_orbitals.
template <typename Emit>
__device__ __forceinline__ void eval_phigrad_f32(const SpecSh &S, const float4 *__restrict__ coef, float dx, float dy,
                                                 float dz, Emit &&emit)
{
    const float r2 = dx * dx + dy * dy + dz * dz;
    const int nrad = S.nrad;
    if (!(r2 < S.rcut2)) {
        int o = 0;
        for (int ir = 0; ir < nrad; ++ir) {
            const int nm = 2 * ((S.lpack >> (2 * ir)) & 3) + 1;
            for (int m = 0; m < nm; ++m, ++o) emit(o, 0.f, 0.f, 0.f, 0.f);
        }
        return;
    }
    if (r2 < 1e-24f) {
        int o = 0;
        for (int ir = 0; ir < nrad; ++ir) {
            const int l = (S.lpack >> (2 * ir)) & 3;
            const float4 c = __ldg(coef + S.coef_off + ir);
            if (l == 0) {
                emit(o++, c.x * YC<float>::c0, 0.f, 0.f, 0.f);
            } else if (l == 1) {
                const float g = c.y * S.inv_dr * YC<float>::c1;
                emit(o++, 0.f, 0.f, 0.f, g);
                emit(o++, 0.f, g, 0.f, 0.f);
                emit(o++, 0.f, 0.f, g, 0.f);
            } else {
                for (int m = 0; m < 5; ++m) emit(o++, 0.f, 0.f, 0.f, 0.f);
            }
        }
        return;
    }
    float ir1 = rsqrtf(r2);
    ir1 = ir1 * (1.5f - 0.5f * r2 * ir1 * ir1);
    const float r = r2 * ir1;
    const float x = r * S.inv_dr;
    int i = (int)x;
    i = min(i, S.nint - 1);
    const float t = x - (float)i;
    const float ux = dx * ir1, uy = dy * ir1, uz = dz * ir1;
    const float4 *cp = coef + S.coef_off + i * nrad;
    int o = 0;
    auto radial = [&](const float4 &c, int ir) {
        const float f = c.x + t * (c.y + t * (c.z + t * c.w));
        const float df = (c.y + t * (2.f * c.z + 3.f * t * c.w)) * S.inv_dr;
        const int l = (S.lpack >> (2 * ir)) & 3;
        if (l == 0) {
            const float a = df * YC<float>::c0;
            emit(o, f * YC<float>::c0, a * ux, a * uy, a * uz);
            o += 1;
        } else if (l == 1) {
            // phi = g S, g = f/r, S = c1 (z, x, y); grad = g' u S + g grad S, g' = (f' - g)/r
            const float g = f * ir1;
            const float gp = (df - g) * ir1;
            const float c1 = YC<float>::c1;
            const float gc = g * c1;
            const float Sz = c1 * dz, Sx = c1 * dx, Sy = c1 * dy;
            emit(o, g * Sz, gp * ux * Sz, gp * uy * Sz, gp * uz * Sz + gc);
            emit(o + 1, g * Sx, gp * ux * Sx + gc, gp * uy * Sx, gp * uz * Sx);
            emit(o + 2, g * Sy, gp * ux * Sy, gp * uy * Sy + gc, gp * uz * Sy);
            o += 3;
        } else {
            const float g = f * ir1 * ir1;
            const float gp = (df - 2.f * f * ir1) * ir1 * ir1;
            const float c20 = YC<float>::c20, c21 = YC<float>::c21, c22 = YC<float>::c22;
            float Sv = c20 * (2.f * dz * dz - dx * dx - dy * dy);
            emit(o, g * Sv, gp * ux * Sv - 2.f * g * c20 * dx, gp * uy * Sv - 2.f * g * c20 * dy,
                 gp * uz * Sv + 4.f * g * c20 * dz);
            Sv = c21 * dx * dz;
            emit(o + 1, g * Sv, gp * ux * Sv + g * c21 * dz, gp * uy * Sv, gp * uz * Sv + g * c21 * dx);
            Sv = c21 * dy * dz;
            emit(o + 2, g * Sv, gp * ux * Sv, gp * uy * Sv + g * c21 * dz, gp * uz * Sv + g * c21 * dy);
            Sv = c22 * (dx * dx - dy * dy);
            emit(o + 3, g * Sv, gp * ux * Sv + 2.f * g * c22 * dx, gp * uy * Sv - 2.f * g * c22 * dy, gp * uz * Sv);
            Sv = c21 * dx * dy;
            emit(o + 4, g * Sv, gp * ux * Sv + g * c21 * dy, gp * uy * Sv + g * c21 * dx, gp * uz * Sv);
            o += 5;
        }
    };
    for (int ir = 0; ir < nrad; ++ir) radial(__ldg(cp + ir), ir);
}

// Density and gradient of one atom image's orbital combination at displacement d:
//   rho += Sum_o phi_o(d) c(o),   (gx, gy, gz) += Sum_o grad phi_o(d) c(o)   (GRAD only)
// for coefficients c(o) (the density-matrix contraction Psi of the point).  Written per radial
// with phi = g(r) S_lm(d), g = f / r^l and S_lm the solid harmonics, so that
//   Sum_m c_m grad phi_m = g'(r) u P + g grad P,   P = Sum_m c_m S_lm(d),
// with grad P linear in d (l <= 2): one radial derivative per radial instead of one gradient per
// orbital.  The caller has checked |d| < rcut.  Same conventions as eval_orbitals (the centre
// limits included).
template <bool GRAD, typename Coeff>
__device__ __forceinline__ void eval_rho_grad_f32(const SpecSh &S, const float4 *__restrict__ coef, float dx,
                                                  float dy, float dz, Coeff &&c, float &rho, float &gx, float &gy,
                                                  float &gz)
{
    const float r2 = dx * dx + dy * dy + dz * dz;
    const int nrad = S.nrad;
    int o = 0;
    if (r2 < 1e-24f) {
        for (int ir = 0; ir < nrad; ++ir) {
            const int l = (S.lpack >> (2 * ir)) & 3;
            const float4 q = __ldg(coef + S.coef_off + ir);
            if (l == 0) {
                rho += q.x * YC<float>::c0 * c(o);
                o += 1;
            } else if (l == 1) {
                if (GRAD) {
                    const float g = q.y * S.inv_dr * YC<float>::c1;   // grad phi_1m = f'(0) c1 e_m
                    gz += g * c(o);
                    gx += g * c(o + 1);
                    gy += g * c(o + 2);
                }
                o += 3;
            } else {
                o += 5;
            }
        }
        return;
    }
    float ir1 = rsqrtf(r2);
    ir1 = ir1 * (1.5f - 0.5f * r2 * ir1 * ir1);
    const float r = r2 * ir1;
    const float x = r * S.inv_dr;
    int i = (int)x;
    i = min(i, S.nint - 1);
    const float t = x - (float)i;
    const float ux = dx * ir1, uy = dy * ir1, uz = dz * ir1;
    const float4 *cp = coef + S.coef_off + i * nrad;
    for (int ir = 0; ir < nrad; ++ir) {
        const float4 q = __ldg(cp + ir);
        const float f = q.x + t * (q.y + t * (q.z + t * q.w));
        const int l = (S.lpack >> (2 * ir)) & 3;
        if (l == 0) {
            const float c0 = c(o) * YC<float>::c0;
            rho += f * c0;
            if (GRAD) {
                const float a = (q.y + t * (2.f * q.z + 3.f * t * q.w)) * S.inv_dr * c0;
                gx += a * ux;
                gy += a * uy;
                gz += a * uz;
            }
            o += 1;
        } else if (l == 1) {
            const float k1 = YC<float>::c1;
            const float Cz = c(o) * k1, Cx = c(o + 1) * k1, Cy = c(o + 2) * k1;
            const float Pv = Cz * dz + Cx * dx + Cy * dy;
            const float g = f * ir1;
            rho += g * Pv;
            if (GRAD) {
                const float df = (q.y + t * (2.f * q.z + 3.f * t * q.w)) * S.inv_dr;
                const float gp = (df - g) * ir1 * Pv;
                gx += gp * ux + g * Cx;
                gy += gp * uy + g * Cy;
                gz += gp * uz + g * Cz;
            }
            o += 3;
        } else {
            const float C0 = c(o) * YC<float>::c20, C1 = c(o + 1) * YC<float>::c21, C2 = c(o + 2) * YC<float>::c21;
            const float C3 = c(o + 3) * YC<float>::c22, C4 = c(o + 4) * YC<float>::c21;
            const float xx = dx * dx, yy = dy * dy, zz = dz * dz;
            const float Pv = C0 * (2.f * zz - xx - yy) + C1 * dx * dz + C2 * dy * dz + C3 * (xx - yy) + C4 * dx * dy;
            const float g = f * ir1 * ir1;
            rho += g * Pv;
            if (GRAD) {
                const float df = (q.y + t * (2.f * q.z + 3.f * t * q.w)) * S.inv_dr;
                const float gp = (df - 2.f * f * ir1) * ir1 * ir1 * Pv;
                const float px = 2.f * (C3 - C0) * dx + C1 * dz + C4 * dy;
                const float py = -2.f * (C0 + C3) * dy + C2 * dz + C4 * dx;
                const float pz = 4.f * C0 * dz + C1 * dx + C2 * dy;
                gx += gp * ux + g * px;
                gy += gp * uy + g * py;
                gz += gp * uz + g * pz;
            }
            o += 5;
        }
    }
}

// eval_rho_grad_f32 for a compiled radial list: all spline records fetched together, the
// radials evaluated side by side
template <class SH, bool GRAD, typename Coeff>
__device__ __forceinline__ void eval_rho_grad_shape(const SpecSh &S, const float4 *__restrict__ coef, float dx,
                                                    float dy, float dz, Coeff &&c, float &rho, float &gx, float &gy,
                                                    float &gz)
{
    const float r2 = dx * dx + dy * dy + dz * dz;
    if (r2 < 1e-24f) {
        eval_rho_grad_f32<GRAD>(S, coef, dx, dy, dz, c, rho, gx, gy, gz);
        return;
    }
    float ir1 = rsqrtf(r2);
    ir1 = ir1 * (1.5f - 0.5f * r2 * ir1 * ir1);
    const float x = r2 * ir1 * S.inv_dr;
    const int i = min((int)x, S.nint - 1);
    const float t = x - (float)i;
    const float4 *cp = coef + S.coef_off + i * SH::nrad;
    float4 q[SH::nrad];
#pragma unroll
    for (int ir = 0; ir < SH::nrad; ++ir) q[ir] = __ldg(cp + ir);
    const float ux = dx * ir1, uy = dy * ir1, uz = dz * ir1;
    const float xx = dx * dx, yy = dy * dy, zz = dz * dz;
    int o = 0;
#pragma unroll
    for (int ir = 0; ir < SH::nrad; ++ir) {
        const float f = q[ir].x + t * (q[ir].y + t * (q[ir].z + t * q[ir].w));
        const float df = (q[ir].y + t * (2.f * q[ir].z + 3.f * t * q[ir].w)) * S.inv_dr;
        if (SH::l(ir) == 0) {
            const float c0 = c(o) * YC<float>::c0;
            rho += f * c0;
            if (GRAD) {
                const float a = df * c0;
                gx += a * ux; gy += a * uy; gz += a * uz;
            }
        } else if (SH::l(ir) == 1) {
            const float k1 = YC<float>::c1;
            const float Cz = c(o) * k1, Cx = c(o + 1) * k1, Cy = c(o + 2) * k1;
            const float Pv = Cz * dz + Cx * dx + Cy * dy;
            const float g = f * ir1;
            rho += g * Pv;
            if (GRAD) {
                const float gp = (df - g) * ir1 * Pv;
                gx += gp * ux + g * Cx; gy += gp * uy + g * Cy; gz += gp * uz + g * Cz;
            }
        } else {
            const float C0 = c(o) * YC<float>::c20, C1 = c(o + 1) * YC<float>::c21, C2 = c(o + 2) * YC<float>::c21;
            const float C3 = c(o + 3) * YC<float>::c22, C4 = c(o + 4) * YC<float>::c21;
            const float Pv = C0 * (2.f * zz - xx - yy) + C1 * dx * dz + C2 * dy * dz + C3 * (xx - yy) + C4 * dx * dy;
            const float g = f * ir1 * ir1;
            rho += g * Pv;
            if (GRAD) {
                const float gp = (df - 2.f * f * ir1) * ir1 * ir1 * Pv;
                gx += gp * ux + g * (2.f * (C3 - C0) * dx + C1 * dz + C4 * dy);
                gy += gp * uy + g * (-2.f * (C0 + C3) * dy + C2 * dz + C4 * dx);
                gz += gp * uz + g * (4.f * C0 * dz + C1 * dx + C2 * dy);
            }
        }
        o += 2 * SH::l(ir) + 1;
    }
}

template <bool GRAD, typename Coeff>
__device__ __forceinline__ void eval_rho_grad_any(const SpecSh &S, const float4 *__restrict__ coef, float dx, float dy,
                                                  float dz, Coeff &&c, float &rho, float &gx, float &gy, float &gz)
{
    if (S.shape == kShapeSPD) eval_rho_grad_shape<ShapeSPD, GRAD>(S, coef, dx, dy, dz, c, rho, gx, gy, gz);
    else if (S.shape == kShapeSP) eval_rho_grad_shape<ShapeSP, GRAD>(S, coef, dx, dy, dz, c, rho, gx, gy, gz);
    else eval_rho_grad_f32<GRAD>(S, coef, dx, dy, dz, c, rho, gx, gy, gz);
}

// ----------------------------------------------------------------------- status and waits
__device__ __forceinline__ void report_timeout(const Plan &P) { atomicCAS(P.status, 0, (int)GINT_ETIMEOUT); }

__device__ __forceinline__ bool aborted(const Plan &P)
{
    return *(volatile int *)P.status != 0;
}

}  // namespace gint
