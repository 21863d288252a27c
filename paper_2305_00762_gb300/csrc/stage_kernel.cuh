// Fused MEG7-prim residual + TVD-RK3 stage update for sm_103a.
//
// One CTA owns a BX x BY tile of interior cells. It stages the tile plus a
// 6-cell halo of the conservative state in shared memory as primitive
// variables, computes every per-cell quantity once (sixth-order gradients in
// x and y, detector flags, cell fluxes), evaluates every x and y face of the
// tile once (characteristic MEG7 states, flux reconstruction, HLLC, viscous
// flux), differences the face fluxes into the residual and applies the stage
// update in FP64. References are to arXiv:2305.00762.
//
// T is the arithmetic type of the stencil, reconstruction and flux work
// (double, or float for the FP32 form); the state, the stage combination and
// the positivity check are always FP64.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fp_convert.cuh"
#include "gbr_internal.h"
#include "sensor.cuh"

namespace gbr {

template <int BX, int BY, bool VISC, bool CONS = false, bool FLUX0 = false>
struct TileLayout {
    static constexpr int V = VISC ? 1 : 0;
    static constexpr int RW = BX + 12, RH = BY + 12;  // staged region (tile + halo)
    static constexpr int NU = RW * RH;
    // The cells any later phase reads: the staged region without its four
    // C x C corners (face stencils run along rows or columns of the tile).
    // C = 6 - V: the viscous tangential gradients reach one row / column
    // further. The learned sensor's direction assignment runs each
    // direction's plain test on the whole detector box [3, B + 9), which
    // reaches the cells [3, 6) of the corners: C = 3 there; its fused
    // inference reads the 5 x 5 windows of the box, [1, B + 11): C = 1.
    template <int LEARNED>
    struct Cross {
        static constexpr int C = LEARNED == 2 ? 1 : (LEARNED ? 3 : 6 - V);
        static constexpr int NMID = RW * (RH - 2 * C), NCOL = RW - 2 * C;
        static constexpr int N = NMID + 2 * C * NCOL;
        // Cross cell e < N is region cell cell(e): first the full-width rows
        // [C, RH - C), then the columns [C, RW - C) of the bottom and top
        // bands of C rows.
        __device__ static __forceinline__ int cell(int e)
        {
            if (e < NMID) return C * RW + e;
            const int f = e - NMID;
            const int band = f / (C * NCOL), g = f - band * (C * NCOL);
            const int r = g / NCOL;
            return (band ? RH - C + r : r) * RW + C + (g - r * NCOL);
        }
    };
    // x-gradients: rows [6-V, 6+BY+V), region columns [3, BX+9)
    static constexpr int GXW = BX + 6, GXH = BY + 2 * V, NGX = GXW * GXH;
    // y-gradients: region rows [3, BY+9), columns [6-V, 6+BX+V)
    static constexpr int GYW = BX + 2 * V, GYH = BY + 6, NGY = GYW * GYH;
    // detector flags: x at interior rows, columns [3, BX+9); y at rows [3, BY+9)
    static constexpr int PXW = BX + 6, NPX = PXW * BY;
    static constexpr int PYH = BY + 6, NPY = PYH * BX;
    // cell fluxes: x at interior rows, columns [1, BX+11); y at rows [1, BY+11)
    static constexpr int FXW = BX + 10, NFX = FXW * BY;
    static constexpr int FYH = BY + 10, NFY = FYH * BX;
    // face fluxes
    static constexpr int HXW = BX + 1, NHX = HXW * BY;
    static constexpr int HYH = BY + 1, NHY = HYH * BX;

    static constexpr int NF = NHX + NHY;  // faces of the tile

    // FLUX0: the cell fluxes are written in phase 0, from the staged
    // conservative values; their arrays then come before the gradients, so
    // that the TMA landing area (at the gradients, over the face fluxes) does
    // not overlap them.
    static constexpr int oU = 0;
    static constexpr int oGX = FLUX0 ? oU + 4 * NU + 4 * (NFX + NFY) : oU + 4 * NU;
    static constexpr int oGY = oGX + 4 * NGX;
    static constexpr int oFX = FLUX0 ? oU + 4 * NU : oGY + 4 * NGY;
    static constexpr int oFY = oFX + 4 * NFX;
    static constexpr int oHX = FLUX0 ? oGY + 4 * NGY : oFY + 4 * NFY;
    static constexpr int oHY = oHX + 4 * NHX;
    static constexpr int oQc = oHY + 4 * NHY;         // conservative values (MEG7-cons)
    static constexpr int oEnd = oQc + (CONS ? 4 * NU : 0);

    // learned sensor: per-cell decisions on the bounding box of both
    // detector regions, rows and columns [3, B+9)
    static constexpr int BOXW = BX + 6, BOXH = BY + 6, NBOX = BOXW * BOXH;

    template <typename T, int NT>
    static constexpr int nT() { return oEnd; }  // elements of T
    template <typename T, int NT>
    static constexpr size_t bytes() { return sizeof(T) * (size_t)nT<T, NT>() + (size_t)(NPX + NPY) + 16; }
    template <typename T, int NT, bool LEARNED>
    static constexpr size_t total_bytes()
    {
        return LEARNED ? (bytes<T, NT>() + NBOX + 15) / 16 * 16 : bytes<T, NT>();
    }

    // TMA staging: the FP64 conservative tile + halo lands as [4][RH][RW]
    // doubles on top of the gradient, face-flux and (without FLUX0)
    // cell-flux arrays, all first written after phase 0, and below the
    // MEG7-cons copy that phase 0 fills.
    static constexpr size_t kRawBytes = sizeof(double) * 4 * (size_t)NU;
    template <typename T>
    static constexpr size_t raw_offset() { return sizeof(T) * (size_t)oGX; }
    template <typename T>
    static constexpr size_t raw_limit() { return sizeof(T) * (size_t)(CONS ? oQc : oEnd); }
};

template <typename T>
__device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }
template <typename T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
// FP32: one min / max instruction (the same value for operands that are not NaN)
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double trsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float trsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double tsinpi(double x) { return sinpi(x); }
__device__ __forceinline__ float tsinpi(float x) { return sinpif(x); }
__device__ __forceinline__ double tabs(double x) { return fabs(x); }
__device__ __forceinline__ float tabs(float x) { return fabsf(x); }

// FP64 comparisons on the integer pipe. GB300 runs every FP64 instruction,
// compares and min/max included, on a unit that retires 2 thread-operations
// per SM per clock, against 64 for the 32-bit integer pipe; the MP limiter is
// mostly comparisons. For doubles that are not NaN, the signed 64-bit order of
// ordkey(x) is the order of x (with -0 just below +0), ordkey is its own
// inverse, and |x| orders as the bit pattern of x with the sign cleared.
// Values chosen this way equal those of the floating-point comparisons; only
// the sign of a zero result may differ, which no later sum or product turns
// into a different non-zero value.
__device__ __forceinline__ long long ordkey(double x)
{
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ double tmin(double a, double b) { return ordkey(a) < ordkey(b) ? a : b; }
__device__ __forceinline__ double tmax(double a, double b) { return ordkey(a) > ordkey(b) ? a : b; }

// Eq. alpha: minmod(a, b) = 1/2 (sign a + sign b) min(|a|, |b|): the operand
// of smaller magnitude when the signs agree, else 0. FP32: that is the
// median of a, b and 0, four min / max instructions; FP64: the sign test on
// the bits and the magnitudes compared as integers. Only the sign of a zero
// result may differ from the formula's.
__device__ __forceinline__ float minmod(float a, float b)
{
    return fmaxf(fminf(a, b), fminf(fmaxf(a, b), 0.f));
}
__device__ __forceinline__ double minmod(double a, double b)
{
    const long long ba = __double_as_longlong(a), bb = __double_as_longlong(b);
    const unsigned long long ma = (unsigned long long)ba & 0x7FFFFFFFFFFFFFFFULL;
    const unsigned long long mb = (unsigned long long)bb & 0x7FFFFFFFFFFFFFFFULL;
    const double r = ma <= mb ? a : b;  // the smaller magnitude
    return (ba ^ bb) < 0 ? 0.0 : r;     // opposite signs
}

// The MP test's comparison x <= thr (Eq. mp5Condition: 1e-40 for a field in
// the paper's scaling, 1e-40 s^2 for one carried scaled by s; grb_mp tests
// a multiple of the product and scales thr alike).
template <typename T>
__device__ __forceinline__ bool mp_accept(T x, T thr) { return x <= thr; }
__device__ __forceinline__ bool mp_accept(double x, double thr) { return ordkey(x) <= ordkey(thr); }

// The last step of Eq. mp-procedure from Phi_j, Phi_{j+1}, Phi^MD, Phi^UL,
// Phi^LC and the GRB value pl. Phi^min = max(min(Phi_j, Phi_{j+1}, MD),
// min(Phi_j, UL, LC)) is min(Phi_j, max(min(Phi_{j+1}, MD), min(UL, LC)))
// (min distributes over max), and likewise Phi^max: four comparisons each
// instead of five. Phi^min <= Phi_j <= Phi^max, so pl + minmod(Phi^min - pl,
// Phi^max - pl) is the median of pl, Phi^min and Phi^max: pl clamped to
// [Phi^min, Phi^max], taken without arithmetic (the formula's value up to
// the rounding of (Phi^min - pl) + pl).
template <typename T>
__device__ __forceinline__ T mp_clamp(T p2, T p3, T md, T ul, T lc, T pl)
{
    const T pmin = tmin(p2, tmax(tmin(p3, md), tmin(ul, lc)));
    const T pmax = tmax(p2, tmin(tmax(p3, md), tmax(ul, lc)));
    return tmin(tmax(pl, pmin), pmax);
}
// FP32: the bounds as the paper writes them, each a maximum (minimum) of two
// three-operand minima (maxima), the min / max instructions taking three
// operands.
__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float mp_clamp(float p2, float p3, float md, float ul, float lc, float pl)
{
    const float pmin = fmaxf(fmin3(p2, p3, md), fmin3(p2, ul, lc));
    const float pmax = fminf(fmax3(p2, p3, md), fmax3(p2, ul, lc));
    return fminf(fmaxf(pl, pmin), pmax);
}
__device__ __forceinline__ double mp_clamp(double p2, double p3, double md, double ul, double lc, double pl)
{
    const long long k2 = ordkey(p2), k3 = ordkey(p3), km = ordkey(md), ku = ordkey(ul), kl = ordkey(lc);
    const long long kmin = min(k2, max(min(k3, km), min(ku, kl)));
    const long long kmax = max(k2, min(max(k3, km), max(ku, kl)));
    const long long k = min(max(ordkey(pl), kmin), kmax);
    return __longlong_as_double(k ^ ((k >> 63) & 0x7FFFFFFFFFFFFFFFLL));
}

// Explicitly rounded products and fused multiply-adds. Per-cell work that is
// done once along x and once along y sits at two call sites, where the
// compiler could contract a*b + c into an FMA at one and not at the other.
// Written with these, both sites round alike, so the x and y results of
// mirrored data are bitwise mirrors (the face work shares one call site).
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
// a^2 + b^2, symmetric in a and b to the last bit.
template <typename T>
__device__ __forceinline__ T sumsq(T a, T b) { return rmul(a, a) + rmul(b, b); }

// Eq. pressure: primitives (rho, u, v, p) of a conservative state, in T,
// rounded alike wherever it is inlined (the stage kernels' staging and the
// learned sensor's).
template <typename T>
__device__ __forceinline__ void prims_of(double q0, double q1, double q2, double q3, T gm1, T& r, T& u, T& v, T& p)
{
    r = from_f64<T>(q0);
    const T ir = T(1) / r;
    u = from_f64<T>(q1) * ir;
    v = from_f64<T>(q2) * ir;
    p = gm1 * rfma(-rmul(T(0.5), r), sumsq(u, v), from_f64<T>(q3));
}

// Sec. 2.5: CFL wavespeed of one cell state, max((|u| + c)/dx, (|v| + c)/dy)
// (and the viscous bound 4 nu / dx^2 when mu > 0), in T. Every operation is
// contraction-free or explicitly rounded, so the stage epilogue and the
// standalone reduction give the same bits (a resumed run picks the same dt).
template <typename T>
__device__ __forceinline__ T cell_wavespeed_t(double q0, double q1, double q2, double q3, T gamma, T gm1, T mu,
                                              T inv_dx, T inv_dy)
{
    T r, u, v, p;
    prims_of(q0, q1, q2, q3, gm1, r, u, v, p);
    const T ir = T(1) / r;
    const T cs = tsqrt(gamma * p * ir);
    T l = tmax((tabs(u) + cs) * inv_dx, (tabs(v) + cs) * inv_dy);
    if (mu > T(0)) {
        const T nu4 = T(4) * mu * ir;
        l = tmax(l, tmax(nu4 * inv_dx * inv_dx, nu4 * inv_dy * inv_dy));
    }
    return l;
}
template <typename T>
__device__ __forceinline__ double cell_wavespeed(double q0, double q1, double q2, double q3, T gamma, T gm1, T mu,
                                                 T inv_dx, T inv_dy)
{
    return to_f64(cell_wavespeed_t<T>(q0, q1, q2, q3, gamma, gm1, mu, inv_dx, inv_dy));
}
// max with fmax semantics (a NaN operand is ignored), in T
__device__ __forceinline__ double tmax_nan(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float tmax_nan(float a, float b) { return fmaxf(a, b); }

// IEEE predicates of an FP64 value from its bits (integer pipes):
// finite, and 0 < x (NaN excluded, +inf included).
__device__ __forceinline__ bool finite_bits(double x) { return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000; }
__device__ __forceinline__ bool positive_bits(double x)
{
    const long long b = __double_as_longlong(x);
    return b > 0 && b <= 0x7ff0000000000000LL;
}
// 0 < x in T: the comparison itself in FP32, the bit test in FP64 (off the
// FP64 pipe; the same answer for every value, NaN included).
__device__ __forceinline__ bool tpositive(float x) { return x > 0.0f; }
__device__ __forceinline__ bool tpositive(double x) { return positive_bits(x); }
// a < b for values that are not NaN, in T (FP64 on the integer pipe).
__device__ __forceinline__ bool tless(float a, float b) { return a < b; }
__device__ __forceinline__ bool tless(double a, double b) { return ordkey(a) < ordkey(b); }

// Eq. six: the dx-scaled sixth-order gradient at s[0] along stride st,
// carried as 60 times its value (45 D1 - 9 D2 + D3, without the final
// division): every consumer is linear in the gradients and takes the 1/60
// into its own constant factors (kGrad below).
template <typename T>
__device__ __forceinline__ T grad6(const T* s, int st)
{
    return rfma(T(45), s[st] - s[-st], rfma(T(-9), s[2 * st] - s[-2 * st], s[3 * st] - s[-3 * st]));
}
constexpr double kGrad = 60.0;  // the scale of the carried gradients

// Eq. detector with eps = 0.9 psi_c xi^2 / (1 - 0.9 psi_c), xi = 1e-3: returns
// true when psi_j < psi_c = 0.5. psi = (2ab + eps)/(a^2 + b^2 + eps) and the
// denominator is positive, so psi < 1/2 <=> 2 (2ab + eps) < a^2 + b^2 + eps.
template <typename T>
__device__ __forceinline__ bool trouble_cell(const T* r, int st)
{
    const T eps = T(0.9 * 0.5 / (1.0 - 0.9 * 0.5) * 1e-6);
    const T a = tabs(r[0] - r[-st]) + tabs(rfma(T(-2), r[-st], r[0]) + r[-2 * st]);
    const T b = tabs(r[0] - r[st]) + tabs(rfma(T(-2), r[st], r[0]) + r[2 * st]);
    return tless(T(2) * rfma(T(2) * a, b, eps), rfma(a, a, rfma(b, b, eps)));
}

// The value of psi itself (Eq. detector), same a, b and eps as trouble_cell.
__device__ __forceinline__ double detector_psi(const double* r, int st)
{
    const double eps = 0.9 * 0.5 / (1.0 - 0.9 * 0.5) * 1e-6;
    const double a = fabs(r[0] - r[-st]) + fabs(rfma(-2.0, r[-st], r[0]) + r[-2 * st]);
    const double b = fabs(r[0] - r[st]) + fabs(rfma(-2.0, r[st], r[0]) + r[2 * st]);
    return rfma(2.0 * a, b, eps) / rfma(a, a, rfma(b, b, eps));
}

// The GRB left value and the MP test of Eqs. mp5Condition and alpha for the left value
// at j+1/2 from Phi_{j-2..j+2} (p[0..4]) and Phi'_{j-2..j+2} (d[0..4]),
// xi = 7. Returns the GRB value; `need` is set when the MP limiter must be
// applied. The GRB weights of Phi sum to one (478 + 2*178 + 2*3 = 840), so
// Eq. grb is evaluated as Phi_j plus weighted differences: on flat data Phi^L
// equals Phi_j exactly and the test passes (the limiter would return Phi_j).
// Weights of the left value Phi_j + (w0 Phi'_j + w1 (Phi'_{j-1} - Phi'_{j+1})
// + w2 (D_{-1} + D_{+1}) + w3 (D_{-2} + D_{+2})) / 840 with D_k = Phi_{j+k} -
// Phi_j, and of 1/2 (F(f_L) + F(f_R)) = sum_k c_k (f_{j+1-k} + f_{j+k}) / den.
// Order 7: Eq. grb and Eqs. flux-full/flux-right. Order 4 (alpha = 4,
// beta = 0 in Eqs. good_6tth-order_scheme_flux and alpha-beta):
// Phi^L = Phi_j + Phi'_j/2 + (Phi'_{j-1} - Phi'_{j+1})/24 + (D_{-1} + D_{+1})/6,
// and Eq. fourth with its mirror.
template <typename T>
struct GrbCoef {
    T w1, w2, w3;          // w0 = 420 for both orders; the GRB sum takes wk / 840
    T c1, c2, c3, c4, c5;  // pairs (j, j+1), (j-1, j+2), ..., (j-4, j+5)
    T inv_den;
};

template <typename T>
__device__ __forceinline__ GrbCoef<T> grb_coef(int order)
{
    GrbCoef<T> c;
    if (order == 4) {
        c.w1 = T(35);
        c.w2 = T(140);
        c.w3 = T(0);
        c.c1 = T(1821);
        c.c2 = T(-461);
        c.c3 = T(85);
        c.c4 = T(-4);
        c.c5 = T(-1);
        c.inv_den = T(1.0 / 2880.0);
    } else {
        c.w1 = T(60);
        c.w2 = T(178);
        c.w3 = T(3);
        c.c1 = T(1052);
        c.c2 = T(-250);
        c.c3 = T(38);
        c.c4 = T(1);
        c.c5 = T(-1);
        c.inv_den = T(1.0 / 1680.0);
    }
    return c;
}

// In terms of the differences to the centre cell, Dm1 = Phi_{j-1} - Phi_j,
// Dp1 = Phi_{j+1} - Phi_j, S2 = D_{-2} + D_{+2}, and dd = Phi'_{j-1} -
// Phi'_{j+1}: Phi^L = Phi_j + delta with delta the weighted sum above, and
// Phi^MP = Phi_j + m with m = minmod(Dp1, -7 Dm1). The MP test of Eq.
// mp5Condition, (Phi^L - Phi_j)(Phi^L - Phi^MP) <= 1e-40, is taken as
// delta (delta - m) <= 1e-40 (the same quantity, rounded differently; the
// limited value is continuous across the test's boundary, where Phi^L lies
// within the MP bounds). With the gradients at their carried scale kGrad,
// D = 2 kGrad delta has the unit weight on Phi'_j (three FMAs, no product),
// and the test is taken on D: D (D - 2 kGrad m) <= (2 kGrad)^2 1e-40. The
// caller passes Dp1s = 2 kGrad Dp1 and thr = 1e-40 kMP (times the square of
// the field's own scaling, see mp_accept).
constexpr double kGrbD = 2.0 * kGrad;           // D = kGrbD delta
constexpr double kMP = kGrbD * kGrbD;           // the MP threshold's factor
template <typename T>
__device__ __forceinline__ T grb_mp(T pj, T Dm1, T Dp1s, T s1, T S2, T dj, T dd, bool& need, const GrbCoef<T>& C,
                                    T thr)
{
    // the weights times kGrbD / 840 (the gradients' divided by their scale)
    T D = rfma(C.w2 * T(kGrbD / 840.0), s1, rfma(C.w1 * T(2.0 / 840.0), dd, dj));
    if (C.w3 != T(0)) D = rfma(C.w3 * T(kGrbD / 840.0), S2, D);
    const T ms = minmod(Dp1s, T(-7.0 * kGrbD) * Dm1);
    need = !mp_accept(D * (D - ms), thr);
    return rfma(T(1.0 / kGrbD), D, pj);
}

// Eq. mp-procedure: the MP-limited value given the GRB value pl. The
// curvature d_j = 2 (Phi_{j-1} - 2 Phi_j + Phi_{j+1}) - (Phi'_{j+1} -
// Phi'_{j-1})/2 can come from the sums the GRB value was formed with: s1 =
// Dm1 + Dp1 and dd = Phi'_{j-1} - Phi'_{j+1}.
// Its products are explicitly rounded: the packed path of meg7_pair inlines
// it and the per-lane path runs the same arithmetic in mp_limit_pair, and
// the two must round alike.
// The curvature d_{j+1} is the other side's d_j (the right value at the same
// face is centred on cell j+1, mirrored, and the curvature is unchanged by
// the mirror): it comes from that side's sums s1o, ddo.
// The curvatures are carried as 2 kGrad d (one operation fewer each, with
// the gradients at their carried scale; minmod(s a, s b) = s minmod(a, b)
// for s > 0), so Phi^MD and Phi^LC take the factors 1/(2 kGrad) and
// 2/(3 kGrad).
template <typename T>
__device__ __forceinline__ T mp_limit(const T* p, const T* d, T pl, T s1, T dd, T s1o, T ddo)
{
    const T dm1 = rfma(T(4 * kGrad), rfma(T(-2), p[1], p[2]) + p[0], d[0] - d[2]);
    // (d_j and d_{j+1} from the sums: one FMA each)
    const T dj = rfma(T(4 * kGrad), s1, dd);
    const T dp1 = rfma(T(4 * kGrad), s1o, ddo);
    const T md = rmul(T(0.5), rfma(T(-0.5 / kGrad), minmod(dj, dp1), p[2] + p[3]));
    const T Dm1 = p[1] - p[2];
    const T ul = rfma(T(-7), Dm1, p[2]);
    const T lc = rfma(T(2.0 / (3.0 * kGrad)), minmod(dj, dm1), rfma(T(-0.5), Dm1, p[2]));
    return mp_clamp(p[2], p[3], md, ul, lc, pl);
}

// mp_limit for both values of one face and field, where a lane limits its
// own left and right values (w = Phi_{j-2..j+3}, e their gradients; aL, aR,
// s1L, s1R, ddL, ddR as formed for the GRB values). The two sides share
// Phi^MD: the right value's stencil is the left's mirrored about the face,
// so Phi_j + Phi_{j+1} and minmod(d_j, d_{j+1}) are the same for both (the
// sum and minmod are symmetric in their operands), and each side's d_{j+1}
// is the other side's d_j. Every value is bitwise that of mp_limit.
template <typename T>
__device__ __forceinline__ void mp_limit_pair(const T (&w)[6], const T (&e)[6], T aL, T aR, T s1L, T s1R, T ddL,
                                              T ddR, T& vl, T& vr, bool needL, bool needR)
{
    const T djL = rfma(T(4 * kGrad), s1L, ddL), djR = rfma(T(4 * kGrad), s1R, ddR);  // at j and j+1
    const T md = rmul(T(0.5), rfma(T(-0.5 / kGrad), minmod(djL, djR), w[2] + w[3]));
    const T dmL = rfma(T(4 * kGrad), rfma(T(-2), w[1], w[2]) + w[0], e[0] - e[2]);  // at j-1
    const T dmR = rfma(T(4 * kGrad), rfma(T(-2), w[4], w[3]) + w[5], e[3] - e[5]);  // at j+2
    const T ulL = rfma(T(-7), aL, w[2]), ulR = rfma(T(-7), aR, w[3]);
    const T lcL = rfma(T(2.0 / (3.0 * kGrad)), minmod(djL, dmL), rfma(T(-0.5), aL, w[2]));
    const T lcR = rfma(T(2.0 / (3.0 * kGrad)), minmod(djR, dmR), rfma(T(-0.5), aR, w[3]));
    if (needL) vl = mp_clamp(w[2], w[3], md, ulL, lcL, vl);
    if (needR) vr = mp_clamp(w[3], w[2], md, ulR, lcR, vr);
}

// Position of the n-th (0-based) set bit of m; m has more than n set bits.
__device__ __forceinline__ int nth_set_bit(unsigned m, int n)
{
    int pos = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const int c = __popc(m & ((1u << s) - 1u));
        if (n >= c) {
            n -= c;
            m >>= s;
            pos += s;
        }
    }
    return pos;
}

// MEG7 left and right values at face j+1/2 of one characteristic field, from
// its values w[0..5] and gradients e[0..5] at cells j-2..j+3: the left value
// from cells j-2..j+2, the right one from the stencil mirrored about the face
// (cell j+1-k in the place of cell j+k, gradients with their sign changed).
//
// Where the MP test fails (a third of the values or more in developed flow),
// the limiter runs; with one face per lane nearly every warp has such a lane,
// so per lane the limiter would cost the whole warp every time. In FP64, on a
// warp whose left and right failures together number at most 32, the failing
// values are packed onto the warp's lanes instead (each lane fetches one
// stencil by shuffle), limited in one pass and returned by shuffle. Every
// lane of the warp must call this together. The arithmetic of each value is
// unchanged, so the result is the same.
template <typename T>
__device__ __forceinline__ void meg7_pair(const GrbCoef<T>& C, const T (&w)[6], const T (&e)[6], T& vl, T& vr,
                                          T thr = T(1e-40 * kMP))
{
    bool needL, needR;
    // The two sides share the difference w3 - w2 (the left side's D_{+1} is
    // minus the right side's).
    const T b = w[3] - w[2];
    const T aL = w[1] - w[2], aR = w[4] - w[3];
    const T s1L = aL + b, s1R = aR - b;          // second differences at j, j+1
    const T ddL = e[1] - e[3], ddR = e[2] - e[4];  // (mirrored for the right side)
    const T bs = T(kGrbD) * b;
    vl = grb_mp(w[2], aL, bs, s1L, rfma(T(-2), w[2], w[0] + w[4]), e[2], ddL, needL, C, thr);
    vr = grb_mp(w[3], aR, -bs, s1R, rfma(T(-2), w[3], w[5] + w[1]), -e[3], ddR, needR, C, thr);
    if constexpr (sizeof(T) == 8) {
        const unsigned mL = __ballot_sync(0xffffffffu, needL), mR = __ballot_sync(0xffffffffu, needR);
        const int nL = __popc(mL), nR = __popc(mR);
        if (nL + nR <= 32) {  // warp-uniform
            const int lane = threadIdx.x & 31;
            const bool isR = lane >= nL;
            const bool act = lane < nL + nR;
            const int src = !act ? lane : (isR ? nth_set_bit(mR, lane - nL) : nth_set_bit(mL, lane));
            T W[6], E[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                W[k] = __shfl_sync(0xffffffffu, w[k], src);
                E[k] = __shfl_sync(0xffffffffu, e[k], src);
            }
            // (the source lane's left and right values both travel; the
            // receiving lane picks the side it limits)
            const T gl = __shfl_sync(0xffffffffu, vl, src), gr = __shfl_sync(0xffffffffu, vr, src);
            const T sl = __shfl_sync(0xffffffffu, s1L, src), sr = __shfl_sync(0xffffffffu, s1R, src);
            const T dl = __shfl_sync(0xffffffffu, ddL, src), dr = __shfl_sync(0xffffffffu, ddR, src);
            const T g = isR ? gr : gl, s1 = isR ? sr : sl, dd = isR ? dr : dl;
            const T s1o = isR ? sl : sr, ddo = isR ? dl : dr;
            T p[5], d[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                p[k] = isR ? W[5 - k] : W[k];
                d[k] = isR ? -E[5 - k] : E[k];
            }
            const T lim = mp_limit(p, d, g, s1, dd, s1o, ddo);
            const unsigned below = (1u << lane) - 1u;
            const T rl = __shfl_sync(0xffffffffu, lim, __popc(mL & below));
            const T rr = __shfl_sync(0xffffffffu, lim, (nL + __popc(mR & below)) & 31);
            if (needL) vl = rl;
            if (needR) vr = rr;
            return;
        }
    }
    if (needL || needR) mp_limit_pair(w, e, aL, aR, s1L, s1R, ddL, ddR, vl, vr, needL, needR);
}

// 1/2 (F(f_L) + F(f_R)) at the face after cell f[0]: the sum of Eq.
// flux-full and its mirror Eq. flux-right is the symmetric 10-point stencil
// (-1, 1, 38, -250, 1052 | 1052, -250, 38, 1, -1) / 840 over f_{j-4..j+5}.
template <typename T>
__device__ __forceinline__ T recon_mean(const T* f, int s, const GrbCoef<T>& C)
{
    // the weights divided by den (compile-time products): one product, four FMAs
    T acc = rmul(C.c1 * C.inv_den, f[0] + f[s]);
    acc = rfma(C.c2 * C.inv_den, f[-s] + f[2 * s], acc);
    acc = rfma(C.c3 * C.inv_den, f[-2 * s] + f[3 * s], acc);
    acc = rfma(C.c4 * C.inv_den, f[-3 * s] + f[4 * s], acc);
    return rfma(C.c5 * C.inv_den, f[-4 * s] + f[5 * s], acc);
}

template <typename T>
struct FaceIn {
    const T* u[4];  // primitive planes in face-normal order (rho, un, ut, p) at cell j
    int su;
    const T* g[4];  // dx-scaled normal gradients, same order, at cell j
    int sg;
    const unsigned char* tr;  // detector trouble flags at cell j
    int st;
    const T* f[4];  // cell convective fluxes in face-normal order at cell j
    int sf;
    const T* tun;  // tangential derivative (dx-scaled) of un at cell j
    const T* tut;  // ... of ut
    int stq;       // step from cell j to cell j+1 in the tangential arrays
    // MEG7-cons: conservative values (rho, rho un, rho ut, E) at cell j with
    // stride su (the g planes then hold their gradients), and the tangential
    // gradients of rho (tr0); tun / tut then point at those of rho un / rho ut.
    const T* q[4];
    const T* tr0;
};

template <typename T>
struct PhysT {
    T gamma, gm1, igm1, mu, kq;  // kq = mu / (Pr (gamma - 1))
    int lm;                      // 1: shock-stable HLLC-LM dissipation
};

// The whole interface procedure of Secs. 2.1-2.4 at face j+1/2. Returns the
// total flux in face-normal order and the detector flag sigma.
// Projection of a conservative vector q = (rho, rho un, rho ut, E) onto the
// left eigenvectors of the conservative flux Jacobian at the mean state
// (MEG7-cons): with A = b2 q0 - b1 (u q1 + v q2 - q3), b1 = (gamma-1)/c^2,
// b2 = b1 (u^2+v^2)/2 and t = (u q0 - q1)/c, the four rows give
// (A + t)/2, q0 - A, q2 - v q0, (A - t)/2.
template <typename T>
__device__ __forceinline__ void cons_project(T q0, T q1, T q2, T q3, T ub, T vb, T icb, T b1, T b2, T& w0, T& w1,
                                             T& w2, T& w3)
{
    const T A = b2 * q0 - b1 * (ub * q1 + vb * q2 - q3);
    const T t = (ub * q0 - q1) * icb;
    w0 = T(0.5) * (A + t);
    w1 = q0 - A;
    w2 = q2 - vb * q0;
    w3 = T(0.5) * (A - t);
}

template <typename T, bool VISC, int ORDER, bool CONS = false>
__device__ __forceinline__ void face_flux(const FaceIn<T>& in, const PhysT<T>& P, T inv_dn, T inv_dt, T out[4],
                                          bool& smooth)
{
    const GrbCoef<T> coef = grb_coef<T>(ORDER);  // compile-time constants
    // Eq. buffer: sigma = 0 if psi_k < psi_c for any k in j-2..j+3.
    bool tr = false;
#pragma unroll
    for (int k = -2; k <= 3; ++k) tr |= (in.tr[k * in.st] != 0);
    smooth = !tr;

    const int su = in.su, sg = in.sg;
    // Characteristic projection at the arithmetic-mean state.
    // Every factor from one reciprocal square root y = 1/sqrt(gamma p rho):
    // 1/c = rho y, c = gamma p y, 1/(rho c) = y.
    const T rb = T(0.5) * (in.u[0][0] + in.u[0][su]);
    const T pb = T(0.5) * (in.u[3][0] + in.u[3][su]);
    const T gp = P.gamma * pb;
    const T y = trsqrt(gp * rb);
    const T icb = rb * y;            // 1 / c
    const T cb = gp * y;             // c
    const T c2 = cb * cb;            // c^2
    const T ic2 = icb * icb;         // 1 / c^2
    const T be = T(0.5) * ic2;       // 1 / (2 c^2)

    T wL[4], wR[4];
    if constexpr (!CONS) {
        {  // fields 1 and 4 (u - c and u + c) share un and p. They are
           // carried scaled by 2 c^2, as p -/+ rho c un: GRB, the limiter's
           // bounds and its clamp are linear and scale-free, and the MP
           // test's threshold 1e-40 becomes 1e-40 (2 c^2)^2.
            const T rc = rb * cb;  // rho c
            const T thr = T(4e-40 * kMP) * c2 * c2;
            T w0[6], w3[6], e0[6], e3[6];
    #pragma unroll
            for (int k = 0; k < 6; ++k) {
                const int o = (k - 2);
                const T un = in.u[1][o * su], p = in.u[3][o * su];
                w0[k] = rfma(-rc, un, p);
                w3[k] = rfma(rc, un, p);
                const T gu = in.g[1][o * sg], gp = in.g[3][o * sg];
                e0[k] = rfma(-rc, gu, gp);
                e3[k] = rfma(rc, gu, gp);
            }
            meg7_pair(coef, w0, e0, wL[0], wR[0], thr);
            meg7_pair(coef, w3, e3, wL[3], wR[3], thr);
        }
        {  // field 2 (entropy): rho - p / c^2
            T w[6], e[6];
    #pragma unroll
            for (int k = 0; k < 6; ++k) {
                const int o = (k - 2);
                w[k] = rfma(-ic2, in.u[3][o * su], in.u[0][o * su]);
                e[k] = rfma(-ic2, in.g[3][o * sg], in.g[0][o * sg]);
            }
            meg7_pair(coef, w, e, wL[1], wR[1]);
        }
        {  // field 3 (shear): ut
            T w[6], e[6];
    #pragma unroll
            for (int k = 0; k < 6; ++k) {
                const int o = (k - 2);
                w[k] = in.u[2][o * su];
                e[k] = in.g[2][o * sg];
            }
            meg7_pair(coef, w, e, wL[2], wR[2]);
        }
    } else {
        const T ub = T(0.5) * (in.u[1][0] + in.u[1][su]), vb = T(0.5) * (in.u[2][0] + in.u[2][su]);
        const T b1 = P.gm1 * ic2, b2 = T(0.5) * (ub * ub + vb * vb) * b1;
        T w[4][6], e[4][6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int o = (k - 2);
            cons_project(in.q[0][o * su], in.q[1][o * su], in.q[2][o * su], in.q[3][o * su], ub, vb, icb, b1, b2,
                         w[0][k], w[1][k], w[2][k], w[3][k]);
            cons_project(in.g[0][o * sg], in.g[1][o * sg], in.g[2][o * sg], in.g[3][o * sg], ub, vb, icb, b1, b2,
                         e[0][k], e[1][k], e[2][k], e[3][k]);
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            meg7_pair(coef, w[f], e[f], wL[f], wR[f]);
        }
    }
    // Back with the right eigenvectors: to primitive face states (MEG7-prim)
    // or to conservative ones (MEG7-cons).
    T rL, unL, utL, pL, EL, rR, unR, utR, pR, ER;
    T QL[4], QR[4];
    if constexpr (!CONS) {
        // fields 1 and 4 back from their 2 c^2 scaling: with
        // a = w1 + w4, rho = a / (2 c^2) + w2, p = a / 2 and
        // un = (w4 - w1) / (2 rho c)
        const T hrc = T(0.5) * y;  // 1 / (2 rho c): rho c = gamma p rho y = 1 / y
        const T aL03 = wL[0] + wL[3], aR03 = wR[0] + wR[3];
        rL = rfma(be, aL03, wL[1]);
        unL = hrc * (wL[3] - wL[0]);
        utL = wL[2];
        pL = T(0.5) * aL03;
        rR = rfma(be, aR03, wR[1]);
        unR = hrc * (wR[3] - wR[0]);
        utR = wR[2];
        pR = T(0.5) * aR03;
        // positivity fallback: a face state with rho <= 0 or p <= 0 takes the
        // adjacent cell's state (characteristic reconstruction across a
        // strong shock, e.g. the foot of the double Mach reflection)
        if (!(tpositive(rL) && tpositive(pL))) {
            rL = in.u[0][0];
            unL = in.u[1][0];
            utL = in.u[2][0];
            pL = in.u[3][0];
        }
        if (!(tpositive(rR) && tpositive(pR))) {
            rR = in.u[0][su];
            unR = in.u[1][su];
            utR = in.u[2][su];
            pR = in.u[3][su];
        }
        QL[0] = rL;
        QL[1] = rL * unL;
        QL[2] = rL * utL;
        QR[0] = rR;
        QR[1] = rR * unR;
        QR[2] = rR * utR;
        // E = p / (gamma - 1) + (rho un un + rho ut ut) / 2, from the momenta
        EL = rfma(T(0.5), rfma(QL[1], unL, rmul(QL[2], utL)), rmul(pL, P.igm1));
        ER = rfma(T(0.5), rfma(QR[1], unR, rmul(QR[2], utR)), rmul(pR, P.igm1));
        QL[3] = EL;
        QR[3] = ER;
    } else {
        const T ub = T(0.5) * (in.u[1][0] + in.u[1][su]), vb = T(0.5) * (in.u[2][0] + in.u[2][su]);
        const T h2 = T(0.5) * (ub * ub + vb * vb);
        const T Hb = c2 * P.igm1 + h2, uc = ub * cb;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const T* wv = side == 0 ? wL : wR;
            T* Qs = side == 0 ? QL : QR;
            const T S = wv[0] + wv[1] + wv[3];
            Qs[0] = S;
            Qs[1] = ub * S + cb * (wv[3] - wv[0]);
            Qs[2] = vb * S + wv[2];
            Qs[3] = Hb * (wv[0] + wv[3]) + uc * (wv[3] - wv[0]) + h2 * wv[1] + vb * wv[2];
        }
        rL = QL[0];
        EL = QL[3];
        {
            const T ir = T(1) / rL;
            unL = QL[1] * ir;
            utL = QL[2] * ir;
            pL = P.gm1 * (EL - T(0.5) * rL * (unL * unL + utL * utL));
        }
        rR = QR[0];
        ER = QR[3];
        {
            const T ir = T(1) / rR;
            unR = QR[1] * ir;
            utR = QR[2] * ir;
            pR = P.gm1 * (ER - T(0.5) * rR * (unR * unR + utR * utR));
        }
        // positivity fallback (as for MEG7-prim): the adjacent cell's state
        if (!(tpositive(rL) && tpositive(pL))) {
            rL = in.u[0][0];
            unL = in.u[1][0];
            utL = in.u[2][0];
            pL = in.u[3][0];
            EL = pL * P.igm1 + T(0.5) * rL * (unL * unL + utL * utL);
            QL[0] = rL;
            QL[1] = rL * unL;
            QL[2] = rL * utL;
            QL[3] = EL;
        }
        if (!(tpositive(rR) && tpositive(pR))) {
            rR = in.u[0][su];
            unR = in.u[1][su];
            utR = in.u[2][su];
            pR = in.u[3][su];
            ER = pR * P.igm1 + T(0.5) * rR * (unR * unR + utR * utR);
            QR[0] = rR;
            QR[1] = rR * unR;
            QR[2] = rR * utR;
            QR[3] = ER;
        }
    }

    // Central part 1/2 (F_L + F_R) of the hybrid face fluxes (Sec. 2.4):
    // flux reconstruction where sigma = 1, F(Q_L), F(Q_R) where sigma = 0.
    T Fc[4];
    if (smooth) {
#pragma unroll
        for (int m = 0; m < 4; ++m) Fc[m] = recon_mean(in.f[m], in.sf, coef);
    } else {
        Fc[0] = T(0.5) * (QL[1] + QR[1]);
        Fc[1] = T(0.5) * ((QL[1] * unL + pL) + (QR[1] * unR + pR));
        Fc[2] = T(0.5) * (QL[1] * utL + QR[1] * utR);
        Fc[3] = T(0.5) * (unL * (EL + pL) + unR * (ER + pR));
    }

    // HLLC in the form 1/2 (F_L + F_R) - 1/2 |A| (Q_R - Q_L), Eq. Riemann_revisit,
    // with Toro's star states; k (E/rho + (S*-u)(S* + p/(rho (S-u)))) is
    // expanded so that the only divisions are 1/((S_L - S*)(S_R - S*)), S* and
    // the Roe weight.
    {
        // Per side one reciprocal square root y = 1/sqrt(gamma p rho):
        // c = gamma p y, 1/c = rho y, 1/rho = c y.
        const T gpL = P.gamma * pL, gpR = P.gamma * pR;
        const T yL = trsqrt(gpL * rL), yR = trsqrt(gpR * rR);
        const T cL = gpL * yL, cR = gpR * yR;
        const T icL = rL * yL, icR = rR * yR;
        const T irL = cL * yL, irR = cR * yR;
        const T eL = EL * irL, eR = ER * irR;  // E / rho
        const T HL = rfma(pL, irL, eL), HR = rfma(pR, irR, eR);
        // Roe averages (a_L + q a_R) / (1 + q), q = sqrt(rho_R / rho_L)
        const T xq = rR * irL;
        const T q = xq * trsqrt(xq);
        const T oL = T(1) / (T(1) + q);
        const T ut = oL * rfma(q, unR, unL);
        const T vt = oL * rfma(q, utR, utL);
        const T Ht = oL * rfma(q, HR, HL);
        const T c2t = P.gm1 * (Ht - T(0.5) * (ut * ut + vt * vt));
        const T ct = c2t * trsqrt(c2t);
        const T SL = tmin(unL - cL, ut - ct);
        const T SR = tmax(unR + cR, ut + ct);
        const T mL = rL * (SL - unL), mR = rR * (SR - unR);
        // S* = num / den and 1/(S_L - S*), 1/(S_R - S*) from one division:
        // with nL = S_L den - num, nR = S_R den - num and z = 1/(den nL nR),
        // S* = num nL nR z, 1/(S_L - S*) = den^2 nR z, 1/(S_R - S*) = den^2 nL z
        const T num = pR - pL + mL * unL - mR * unR, den = mL - mR;
        const T nL = SL * den - num, nR = SR * den - num;
        const T nLR = nL * nR;
        const T z = T(1) / (den * nLR);
        const T Ss = num * nLR * z;
        const T d2z = den * den * z;
        const T iL = nR * d2z, iR = nL * d2z;  // 1/(S_L - S*), 1/(S_R - S*)
        T aL = tabs(SL), aR = tabs(SR);
        const T aS = tabs(Ss);
        if (P.lm) {
            // Shock-stable HLLC-LM (Fleischmann, Adami and Adams 2020, used by
            // Examples 7 and 8): the acoustic dissipation scaled by
            // phi = sin(pi/2 min(1, Ma / 0.1)), Ma the larger face-normal Mach
            // number of the two face states; phi = 1 leaves HLLC unchanged.
            const T z = tmax(tabs(unL) * icL, tabs(unR) * icR) * T(10);
            if (z < T(1)) {
                const T phi = tsinpi(T(0.5) * z);
                aL *= phi;
                aR *= phi;
            }
        }
        // 1/2 |A| dQ = 1/2 (aL (QsL - QL) + aS (QsR - QsL) + aR (QR - QsR)),
        // regrouped by state: hL QsL + hS QsR - hQL QL + hQR QR. The star
        // states are Q*_K = k_K (1, S*, ut_K, E_K / rho_K + (S* - un_K) S*)
        // + (0, 0, 0, (S* - un_K) p_K / (S_K - S*)), k_K = m_K / (S_K - S*):
        // the factors h / (S_K - S*) and h k are formed once and the star
        // states never built.
        const T hL = T(0.5) * (aL - aS), hS = T(0.5) * (aS - aR), hQL = T(0.5) * aL, hQR = T(0.5) * aR;
        const T giL = hL * iL, giR = hS * iR;
        const T fL = giL * mL, fR = giR * mR;
        const T tL = Ss - unL, tR = Ss - unR;
        out[0] = Fc[0] - fL - fR + hQL * QL[0] - hQR * QR[0];
        out[1] = Fc[1] - (fL + fR) * Ss + hQL * QL[1] - hQR * QR[1];
        out[2] = Fc[2] - fL * utL - fR * utR + hQL * QL[2] - hQR * QR[2];
        out[3] = Fc[3] - fL * (eL + tL * Ss) - giL * (tL * pL) - fR * (eR + tR * Ss) - giR * (tR * pR) +
                 hQL * QL[3] - hQR * QR[3];
    }

    if constexpr (VISC) {
        // Sec. 2.1: alpha-damping (Eq. alphad, alpha_v = 4) on the shared
        // gradients; T = gamma p / rho with T' by the chain rule.
        const T r0 = in.u[0][0], r1 = in.u[0][su];
        const T n0 = in.u[1][0], n1 = in.u[1][su];
        const T t0 = in.u[2][0], t1 = in.u[2][su];
        const T p0 = in.u[3][0], p1 = in.u[3][su];
        T dr0 = in.g[0][0], dr1 = in.g[0][sg];
        T dn0 = in.g[1][0], dn1 = in.g[1][sg];
        T dt0 = in.g[2][0], dt1 = in.g[2][sg];
        T dp0 = in.g[3][0], dp1 = in.g[3][sg];
        const T ir0 = T(1) / r0, ir1 = T(1) / r1;
        if constexpr (CONS) {  // primitive gradients from the conservative ones (chain rule)
            const T k0 = T(0.5) * (n0 * n0 + t0 * t0), k1 = T(0.5) * (n1 * n1 + t1 * t1);
            const T e0 = dp0, e1 = dp1;  // dE
            dp0 = P.gm1 * (e0 - n0 * dn0 - t0 * dt0 + k0 * dr0);
            dp1 = P.gm1 * (e1 - n1 * dn1 - t1 * dt1 + k1 * dr1);
            dn0 = (dn0 - n0 * dr0) * ir0;
            dn1 = (dn1 - n1 * dr1) * ir1;
            dt0 = (dt0 - t0 * dr0) * ir0;
            dt1 = (dt1 - t1 * dr1) * ir1;
        }
        const T T0 = P.gamma * p0 * ir0, T1 = P.gamma * p1 * ir1;
        const T dT0 = P.gamma * (dp0 * ir0 - p0 * dr0 * ir0 * ir0);
        const T dT1 = P.gamma * (dp1 * ir1 - p1 * dr1 * ir1 * ir1);
        // (the gradients, and so T', at their carried scale kGrad)
        const T hg = T(0.5 / kGrad);
        const T un_n = (hg * (dn0 + dn1) + T(2) * (n1 - hg * dn1 - n0 - hg * dn0)) * inv_dn;
        const T ut_n = (hg * (dt0 + dt1) + T(2) * (t1 - hg * dt1 - t0 - hg * dt0)) * inv_dn;
        const T T_n = (hg * (dT0 + dT1) + T(2) * (T1 - hg * dT1 - T0 - hg * dT0)) * inv_dn;
        T gn0 = in.tun[0], gn1 = in.tun[in.stq], gt0 = in.tut[0], gt1 = in.tut[in.stq];
        if constexpr (CONS) {  // tangential derivatives of un, ut from those of rho un, rho ut, rho
            const T ra0 = in.tr0[0], ra1 = in.tr0[in.stq];
            gn0 = (gn0 - n0 * ra0) * ir0;
            gn1 = (gn1 - n1 * ra1) * ir1;
            gt0 = (gt0 - t0 * ra0) * ir0;
            gt1 = (gt1 - t1 * ra1) * ir1;
        }
        const T un_t = hg * (gn0 + gn1) * inv_dt;
        const T ut_t = hg * (gt0 + gt1) * inv_dt;
        const T unf = T(0.5) * (n0 + n1), utf = T(0.5) * (t0 + t1);
        const T tau_nn = T(2.0 / 3.0) * P.mu * (T(2) * un_n - ut_t);
        const T tau_nt = P.mu * (un_t + ut_n);
        const T q_n = -P.kq * T_n;
        out[1] -= tau_nn;
        out[2] -= tau_nt;
        out[3] += -(tau_nn * unf + tau_nt * utf) + q_n;
    }
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One tile of one stage: phases 0-3 for the BX x BY cells whose first cell is
// (tx0, ty0), including the tile's wavespeed max and error word. Shared by
// the single-grid kernel (one CTA per tile) and the persistent batch kernel
// (a CTA walks many tiles of many grids). Starts and ends with all threads
// synchronised, so consecutive calls may reuse the shared memory.
// ---------------------------------------------------------------------------
// Tile staging by the tensor-memory accelerator: one thread issues a 3-D
// tiled bulk copy (x, y, field) of the tile + halo into shared memory, and
// the CTA waits on an mbarrier for its byte count.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Non-blocking test of phase `parity` of the mbarrier.
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for phase 0 of the mbarrier with an iteration limit (about a second);
// false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar)
{
    for (int it = 0; it < (1 << 24); ++it) {
        if (mbar_test(bar, 0)) return true;
        __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// Fifth-generation tensor cores (tcgen05), shared by the learned sensor's
// decision pass (sensor.cu) and the stage kernel's fused inference: matrix
// and instruction descriptors, MMA issue and commit, tensor-memory loads and
// stores of 32 lanes x 16 columns, and a bounded mbarrier wait.
// ---------------------------------------------------------------------------
// Tensor memory of one warpgroup's network rounds: 64 columns, A at [0, 32)
// (layer 1's features, then layer 2's inputs) and D at [32, 64) (the
// accumulators of both layers in turn).
constexpr unsigned kColA = 0, kColD = 32, kColsPerGroup = 64;

__host__ __device__ constexpr int core_index(int n, int k, int kgroups)
{
    return ((n >> 3) * kgroups + (k >> 3)) * 64 + (n & 7) * 8 + (k & 7);
}

// Shared-memory matrix descriptor (no swizzle, K-major core matrices):
// start address, leading byte offset (between core matrices adjacent in K),
// stride byte offset (between adjacent 8-row groups), descriptor version 1.
__device__ __forceinline__ uint64_t tc_smem_desc(const void* p, unsigned lbo, unsigned sbo)
{
    const unsigned a = smem_addr(p);
    return (uint64_t)((a >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulation, BF16 A and B, both
// K-major, N = 32, M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kSensorH >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem d] (+)= A[tmem a] B[desc], issued by one thread.
__device__ __forceinline__ void tc_mma(uint32_t d, uint32_t a, uint64_t bdesc, bool accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
        "r"(a), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate ? 1 : 0)
        : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned long long* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}

// Wait for phase `parity` of the mbarrier: a tight spin first (an MMA round
// trip takes a few hundred cycles), then polls spaced by sleeps, about a
// second in all; false if it gave up.
__device__ __forceinline__ bool mbar_wait_parity_bounded(unsigned long long* bar, unsigned parity)
{
    for (int it = 0; it < (1 << 12); ++it)
        if (mbar_test(bar, parity)) return true;
    for (int it = 0; it < (1 << 24); ++it) {
        if (mbar_test(bar, parity)) return true;
        __nanosleep(64);
    }
    return false;
}


// Error-word bits: 1 = non-physical state, 2 = a bounded wait gave up.
constexpr unsigned kErrNonPhysical = 1u, kErrTimeout = 2u;

// The learned sensor's inference fused into the FP32 stage (learned mode 2):
// the network's decision for every cell of the tile's detector box (region
// cells [3, B + 9) in each direction), from the FP32 primitives the stage
// has just staged (the same values, features, tensor-core rounds and
// thresholds as the separate decision pass, so the same decisions). Scratch:
// `lo` (>= 20 KB, dead until phase 1) holds the 5-wide window maxima and
// minima and the normalisation scales; `hi` (>= 6.5 KB + 128, dead until
// phase 2) the weights in the tensor cores' core-matrix order. Per CTA 128
// tensor-memory columns, allocated here and freed before returning (the
// kernel's shared memory keeps at most two CTAs on an SM: 256 of 512
// columns). Returns false if a bounded wait gave up (uniform over the CTA).
template <int BX, int BY, int NT, bool VISC>
__device__ bool fused_sensor_decisions(const StageParams& P, const float* sU, unsigned char* sT, unsigned char* lo,
                                       unsigned char* hi)
{
    using L = TileLayout<BX, BY, VISC, false>;
    constexpr int RW = L::RW, NU = L::NU, BW = L::BOXW, NB = L::NBOX;
    constexpr int HR = BY + 10;  // region rows [1, BY + 11) of the windows
    constexpr int G = NT / 128;  // warpgroups: the M = 128 rows of each one's MMAs
    static_assert(NT % 128 == 0, "whole warpgroups");
    const int tid = threadIdx.x, warp = tid >> 5;
    float* hrx = reinterpret_cast<float*>(lo);  // [HR][BW] window max of rho, then min; p likewise
    float* hrn = hrx + HR * BW;
    float* hpx = hrn + HR * BW;
    float* hpn = hpx + HR * BW;
    float* scr = hpn + HR * BW;  // [NB] scales
    float* scp = scr + NB;
    unsigned char* hb = hi + ((128u - (smem_addr(hi) & 127u)) & 127u);
    __nv_bfloat16* w1c = reinterpret_cast<__nv_bfloat16*>(hb);
    __nv_bfloat16* w2c = w1c + kSensorH * kSensorK;
    float* b1 = reinterpret_cast<float*>(w2c + kSensorH * kSensorH);
    float* b2 = b1 + kSensorH;
    float* w3 = b2 + kSensorH;
    float* b3 = w3 + kSensorH;
    __shared__ __align__(8) unsigned long long mma_bar;  // never reused for anything else
    __shared__ unsigned tmem_base;
    const SensorDev* w = P.sensor;
    for (int i = tid; i < kSensorH * kSensorK; i += NT) {
        const int n = i / kSensorK, k = i - n * kSensorK;
        w1c[core_index(n, k, kSensorK / 8)] = w->w1t[n * kW1Pitch + k];
    }
    for (int i = tid; i < kSensorH * kSensorH; i += NT) {
        const int n = i / kSensorH, k = i - n * kSensorH;
        w2c[core_index(n, k, kSensorH / 8)] = w->w2t[n * kW2Pitch + k];
    }
    if (tid < kSensorH) {
        b1[tid] = w->b1[tid];
        b2[tid] = w->b2[tid];
        w3[tid] = w->w3[tid];
    }
    if (tid == 0) {
        *b3 = w->b3;
        mbar_init(&mma_bar, 1);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the MMAs read the weights
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(kColsPerGroup * G)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // window maxima and minima over 5 columns (region columns bx + 1 .. bx + 5)
    for (int e = tid; e < HR * BW; e += NT) {
        const int h = e / BW, bx = e - h * BW;
        const float* r = sU + (h + 1) * RW + (bx + 1);
        const float* p = r + 3 * NU;
        float rmx = r[0], rmn = r[0], pmx = p[0], pmn = p[0];
#pragma unroll
        for (int d = 1; d < 5; ++d) {
            rmx = fmaxf(rmx, r[d]);
            rmn = fminf(rmn, r[d]);
            pmx = fmaxf(pmx, p[d]);
            pmn = fminf(pmn, p[d]);
        }
        hrx[e] = rmx;
        hrn[e] = rmn;
        hpx[e] = pmx;
        hpn[e] = pmn;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = tmem_base;
    // ... then over 5 rows: the scales 1/(max_k |q_k - q_c| + floor) of each box cell
    for (int c = tid; c < NB; c += NT) {
        const int by = c / BW, bx = c - by * BW;
        float rmx = hrx[by * BW + bx], rmn = hrn[by * BW + bx], pmx = hpx[by * BW + bx], pmn = hpn[by * BW + bx];
#pragma unroll
        for (int d = 1; d < 5; ++d) {
            const int o = (by + d) * BW + bx;
            rmx = fmaxf(rmx, hrx[o]);
            rmn = fminf(rmn, hrn[o]);
            pmx = fmaxf(pmx, hpx[o]);
            pmn = fminf(pmn, hpn[o]);
        }
        const float rc = sU[(by + 3) * RW + bx + 3], pc = sU[3 * NU + (by + 3) * RW + bx + 3];
        const float mr = fmaxf(0.f, fmaxf(rmx - rc, rc - rmn)), mp = fmaxf(0.f, fmaxf(pmx - pc, pc - pmn));
        scr[c] = 1.f / (mr + kSensorFloor);
        scp[c] = 1.f / (mp + kSensorFloor);
    }
    __syncthreads();
    // this warp's quarter of the lanes, in its warpgroup's columns
    const uint32_t lanes = ((uint32_t)((warp & 3) * 32) << 16) + kColsPerGroup * (uint32_t)(warp >> 2);
    const uint64_t d1 = tc_smem_desc(w1c, 128, 128 * (kSensorK / 8));
    const uint64_t d2 = tc_smem_desc(w2c, 128, 128 * (kSensorH / 8));
    unsigned phase = 0;
    bool ok = true;
    for (int round = 0; round < (NB + NT - 1) / NT && ok; ++round) {
        const int c = round * NT + tid;
        const bool valid = c < NB;
        const int cc = valid ? c : 0;  // a lane past the box works on cell 0 and stores nothing
        const int by = cc / BW, bx = cc - by * BW;
        const float* r = sU + (by + 3) * RW + (bx + 3);
        const float* p = r + 3 * NU;
        const float sr = scr[cc], sp = scp[cc];
#pragma unroll
        for (int half = 0; half < 2; ++half) {  // features 32 half .. 32 half + 31
            uint32_t a[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int k = 32 * half + 2 * j;
                a[j] = pack_bf16(sensor_feature(r, p, RW, sr, sp, k), sensor_feature(r, p, RW, sr, sp, k + 1));
            }
            tc_st16(tm + lanes + kColA + 16 * half, a);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        if (tid == 0 && !(P.stall_mma && round == 0)) {
            tc_fence_after();
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int ks = 0; ks < kSensorK / 16; ++ks)
                    tc_mma(tm + kColsPerGroup * g + kColD, tm + kColsPerGroup * g + kColA + 8 * ks,
                           d1 + (uint64_t)((256 * ks) >> 4), ks > 0);
            tc_commit(&mma_bar);
        }
        bool done = true;
        if (warp == 0) done = mbar_wait_parity_bounded(&mma_bar, phase);
        if (!__syncthreads_and(done)) {
            ok = false;
            break;
        }
        phase ^= 1u;
        tc_fence_after();
        uint32_t hh[16];
#pragma unroll
        for (int half = 0; half < 2; ++half) {  // hidden units 16 half .. 16 half + 15
            uint32_t d[16];
            tc_ld16(tm + lanes + kColD + 16 * half, d);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int n = 16 * half + 2 * j;
                hh[8 * half + j] = pack_bf16(fmaxf(__uint_as_float(d[2 * j]) + b1[n], 0.f),
                                             fmaxf(__uint_as_float(d[2 * j + 1]) + b1[n + 1], 0.f));
            }
        }
        tc_st16(tm + lanes + kColA, hh);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int ks = 0; ks < kSensorH / 16; ++ks)
                    tc_mma(tm + kColsPerGroup * g + kColD, tm + kColsPerGroup * g + kColA + 8 * ks,
                           d2 + (uint64_t)((256 * ks) >> 4), ks > 0);
            tc_commit(&mma_bar);
        }
        done = true;
        if (warp == 0) done = mbar_wait_parity_bounded(&mma_bar, phase);
        if (!__syncthreads_and(done)) {
            ok = false;
            break;
        }
        phase ^= 1u;
        tc_fence_after();
        float z = 0.f;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            uint32_t d[16];
            tc_ld16(tm + lanes + kColD + 16 * half, d);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int n = 16 * half + j;
                z += fmaxf(__uint_as_float(d[j]) + b2[n], 0.f) * w3[n];
            }
        }
        const float pv = 1.f / (1.f + expf(-(z + *b3)));
        if (valid) sT[c] = pv > kSensorHi ? 1 : (pv < kSensorLo ? 0 : 2);
    }
    // release the columns after the last wait (no MMA is in flight: every
    // issued batch was waited for, and a withheld one was never issued)
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(kColsPerGroup * G)
                     : "memory");
    }
    return ok;
}

// LEARNED: 0 = the density detector; 1 = the learned sensor's decisions
// read from the decision pass (P.dec); 2 = the learned sensor's inference
// fused into the stage (FP32 only).
template <typename T, int BX, int BY, int NT, bool VISC, int LEARNED = 0, int ORDER = 7, bool CONS = false,
          bool TMA = false>
__device__ __forceinline__ void stage_tile(const StageParams& P, const int tx0, const int ty0,
                                           unsigned char* smem_raw, const CUtensorMap* tmap = nullptr)
{
    // FP64: the cell fluxes come from the staged conservative values in
    // phase 0 (FLUX0)
    constexpr bool FLUX0 = sizeof(T) == 8;
    using L = TileLayout<BX, BY, VISC, CONS, FLUX0>;
    using X = typename L::template Cross<LEARNED>;  // the staged cells
    T* const sm = reinterpret_cast<T*>(smem_raw);
    T* const sU = sm + L::oU;
    T* const sGX = sm + L::oGX;
    T* const sGY = sm + L::oGY;
    T* const sFX = sm + L::oFX;
    T* const sFY = sm + L::oFY;
    T* const sHX = sm + L::oHX;
    T* const sHY = sm + L::oHY;
    T* const sQc = sm + L::oQc;  // MEG7-cons only
    unsigned char* const sPX = reinterpret_cast<unsigned char*>(sm + L::template nT<T, NT>());
    unsigned char* const sPY = sPX + L::NPX;
    constexpr int RW = L::RW, NU = L::NU, V = L::V;

    const int nx = P.g.nx, ny = P.g.ny, pitch = P.g.pitch;
    const long long plane = P.g.plane;
    const int tid = threadIdx.x;

    PhysT<T> ph;
    ph.gamma = T(P.ph.gamma);
    ph.gm1 = T(P.ph.gm1);
    ph.igm1 = T(P.ph.igm1);
    ph.mu = T(P.ph.mu);
    ph.kq = T(P.ph.kq);
    ph.lm = P.ph.riemann;
    const T inv_dx = T(P.ph.inv_dx), inv_dy = T(P.ph.inv_dy);

    // Phase 0: stage the tile + halo as primitive variables (Eq. pressure).
    // Region cell (rx, ry) is padded cell (tx0 + rx, ty0 + ry).
    auto stage_cell = [&](int idx, double q0, double q1, double q2, double q3) {
        T r, u, v, p;
        prims_of(q0, q1, q2, q3, ph.gm1, r, u, v, p);
        sU[idx] = r;
        sU[NU + idx] = u;
        sU[2 * NU + idx] = v;
        sU[3 * NU + idx] = p;
        if constexpr (FLUX0) {
            // cell fluxes F^c = (rho u, rho u u + p, rho u v, u (E + p)) and
            // G^c (Sec. 1) with rho u, rho v and E taken from the state
            const int ry = idx / RW, rx = idx - ry * RW;
            if (ry >= 6 && ry < 6 + BY && rx >= 1 && rx < BX + 11) {
                const int f = (ry - 6) * L::FXW + (rx - 1);
                sFX[f] = q1;
                sFX[L::NFX + f] = rfma(T(q1), u, p);
                sFX[2 * L::NFX + f] = T(q1) * v;
                sFX[3 * L::NFX + f] = u * (T(q3) + p);
            }
            if (ry >= 1 && ry < BY + 11 && rx >= 6 && rx < BX + 6) {
                const int f = (ry - 1) * BX + (rx - 6);
                sFY[f] = q2;
                sFY[L::NFY + f] = T(q2) * u;
                sFY[2 * L::NFY + f] = rfma(T(q2), v, p);
                sFY[3 * L::NFY + f] = v * (T(q3) + p);
            }
        }
        if constexpr (CONS) {
            sQc[idx] = r;
            sQc[NU + idx] = from_f64<T>(q1);
            sQc[2 * NU + idx] = from_f64<T>(q2);
            sQc[3 * NU + idx] = from_f64<T>(q3);
        }
    };
    bool staged = false;
    if constexpr (TMA) {
        // The whole region in one tensor copy; cells beyond the padded extent
        // (ragged last tiles) read as zero and only feed results that are
        // never stored.
        static_assert(BX % 2 == 0 && L::RW % 2 == 0, "TMA x offsets and rows must be 16-byte multiples");
        static_assert(L::RW <= 256 && L::RH <= 256, "TMA box too large");
        static_assert(L::template raw_offset<T>() + L::kRawBytes <= L::template raw_limit<T>(),
                      "TMA landing area overlaps live shared memory");
        double* raw = reinterpret_cast<double*>(smem_raw + L::template raw_offset<T>());
        __shared__ __align__(8) unsigned long long tma_bar;  // never reused for anything else
        unsigned long long* bar = &tma_bar;
        if ((smem_addr(raw) & 127u) == 0) {  // uniform: the copy needs a 128-byte aligned destination
            if (tid == 0) {
                mbar_init(bar, 1);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            __syncthreads();
            if (tid == 0) {
                mbar_arrive_expect_tx(bar, (unsigned)L::kRawBytes + P.stall_bytes);
                tma_load_3d(raw, tmap, tx0, ty0, 0, bar);
            }
            const bool ok = mbar_wait_bounded(bar);
            if (__syncthreads_or(!ok)) {
                // Give the copy one more bounded wait before the CTA leaves.
                // Leaving is safe only once the copy's bytes have landed: a
                // copy still in flight after this second wait would write
                // into shared memory the SM may have handed to another CTA.
                // The timeout bit set here makes the next synchronising call
                // fail and stays set until gbr_set_state, so no result
                // computed after such an event is reported as valid.
                mbar_wait_bounded(bar);
                if (tid == 0) atomicOr(P.err, kErrTimeout);
                return;
            }
            for (int e = tid; e < X::N; e += NT) {
                const int idx = X::cell(e);
                stage_cell(idx, raw[idx], raw[NU + idx], raw[2 * NU + idx], raw[3 * NU + idx]);
            }
            staged = true;
        }
    }
    if (!staged) {
        // Plain loads, clamped to the padded extent (the clamped cells only
        // feed results that are never stored).
        for (int e = tid; e < X::N; e += NT) {
            const int idx = X::cell(e);
            const int ry = idx / RW, rx = idx - ry * RW;
            const int gx = min(tx0 + rx, nx + 2 * kGhost - 1);
            const int gy = min(ty0 + ry, ny + 2 * kGhost - 1);
            const long long o = (long long)gy * pitch + gx;
            stage_cell(idx, P.q[o], P.q[o + plane], P.q[o + 2 * plane], P.q[o + 3 * plane]);
        }
    }
    if constexpr (LEARNED == 1) {
        // The learned sensor's per-cell decisions (1 = trouble, 0 = smooth,
        // 2 = unsure: the plain detector decides below) of the detector's
        // bounding box, written by the sensor pass for padded cells
        // [3, n + 9) in each direction; box cell (bx, by) is padded cell
        // (tx0 + bx + 3, ty0 + by + 3). Cells past that range (ragged last
        // tiles) only feed results that are never stored.
        unsigned char* const sT = sPY + L::NPY;
        for (int c = tid; c < L::NBOX; c += NT) {
            const int by = c / L::BOXW, bx = c - by * L::BOXW;
            const int gx = min(tx0 + bx + 3, nx + 8), gy = min(ty0 + by + 3, ny + 8);
            sT[c] = P.dec[(long long)gy * pitch + gx];
        }
    }
    __syncthreads();
    if constexpr (LEARNED == 2) {
        static_assert(sizeof(T) == 4, "the fused sensor runs in the FP32 form");
        static_assert(sizeof(T) * (L::oHX - L::oGX) >= sizeof(float) * (4 * (BY + 10) * L::BOXW + 2 * L::NBOX),
                      "fused sensor scratch exceeds the gradient and flux arrays");
        static_assert(sizeof(T) * (L::oQc - L::oHX) >= 128 + 2 * (kSensorH * kSensorK + kSensorH * kSensorH) +
                                                           sizeof(float) * (3 * kSensorH + 1),
                      "fused sensor weights exceed the face-flux arrays");
        unsigned char* const sTd = sPY + L::NPY;
        if (!fused_sensor_decisions<BX, BY, NT, VISC>(P, reinterpret_cast<const float*>(sU), sTd,
                                                      smem_raw + L::template raw_offset<T>(),
                                                      smem_raw + sizeof(T) * L::oHX)) {
            if (tid == 0) atomicOr(P.err, kErrTimeout);
            return;
        }
        __syncthreads();
    }

    // Phase 1: per-cell quantities, each computed once per tile.
    const T* const sV = CONS ? sQc : sU;  // the reconstructed variables
    for (int idx = tid; idx < L::NGX; idx += NT) {  // x-gradients (Eq. six)
        const int a = idx / L::GXW, b = idx - a * L::GXW;
        const T* s = sV + (a + 6 - V) * RW + (b + 3);
#pragma unroll
        for (int m = 0; m < 4; ++m) sGX[m * L::NGX + idx] = grad6(s + m * NU, 1);
    }
    for (int idx = tid; idx < L::NGY; idx += NT) {  // y-gradients
        const int a = idx / L::GYW, b = idx - a * L::GYW;
        const T* s = sV + (a + 3) * RW + (b + 6 - V);
#pragma unroll
        for (int m = 0; m < 4; ++m) sGY[m * L::NGY + idx] = grad6(s + m * NU, RW);
    }
    if constexpr (!LEARNED) {
        for (int idx = tid; idx < L::NPX; idx += NT) {  // x detector (Eq. detector)
            const int a = idx / L::PXW, b = idx - a * L::PXW;
            sPX[idx] = trouble_cell(sU + (a + 6) * RW + (b + 3), 1) ? 1 : 0;
        }
        for (int idx = tid; idx < L::NPY; idx += NT) {  // y detector
            const int a = idx / BX, b = idx - a * BX;
            sPY[idx] = trouble_cell(sU + (a + 3) * RW + (b + 6), RW) ? 1 : 0;
        }
    }
    for (int idx = tid; idx < (FLUX0 ? 0 : L::NFX); idx += NT) {  // cell x-fluxes F^c (Sec. 1)
        const int a = idx / L::FXW, b = idx - a * L::FXW;
        const int c = (a + 6) * RW + (b + 1);
        const T r = sU[c], u = sU[NU + c], v = sU[2 * NU + c], p = sU[3 * NU + c];
        const T E = rfma(p, ph.igm1, rmul(T(0.5) * r, sumsq(u, v)));
        const T ru = r * u;
        sFX[idx] = ru;
        sFX[L::NFX + idx] = rfma(ru, u, p);
        sFX[2 * L::NFX + idx] = ru * v;
        sFX[3 * L::NFX + idx] = u * (E + p);
    }
    for (int idx = tid; idx < (FLUX0 ? 0 : L::NFY); idx += NT) {  // cell y-fluxes G^c
        const int a = idx / BX, b = idx - a * BX;
        const int c = (a + 1) * RW + (b + 6);
        const T r = sU[c], u = sU[NU + c], v = sU[2 * NU + c], p = sU[3 * NU + c];
        const T E = rfma(p, ph.igm1, rmul(T(0.5) * r, sumsq(u, v)));
        const T rv = r * v;
        sFY[idx] = rv;
        sFY[L::NFY + idx] = rv * u;
        sFY[2 * L::NFY + idx] = rfma(rv, v, p);
        sFY[3 * L::NFY + idx] = v * (E + p);
    }
    __syncthreads();
    if constexpr (LEARNED) {
        // Per-direction flags from the sensor's per-cell decision. Smooth (0):
        // no flag. Unsure (2): the plain detector of that direction. Trouble
        // (1): the single output does not say along which axis the jump lies,
        // so the plain tests assign the direction, and a cell neither of them
        // marks keeps the network's flag in both directions.
        const unsigned char* const sT = sPY + L::NPY;
        for (int idx = tid; idx < L::NPX; idx += NT) {
            const int a = idx / L::PXW, b = idx - a * L::PXW;
            const unsigned char d = sT[(a + 3) * L::BOXW + b];
            unsigned char f = 0;
            if (d != 0) {
                const T* c = sU + (a + 6) * RW + (b + 3);
                const bool tx = trouble_cell(c, 1);
                f = (tx || (d == 1 && !trouble_cell(c, RW))) ? 1 : 0;
            }
            sPX[idx] = f;
        }
        for (int idx = tid; idx < L::NPY; idx += NT) {
            const int a = idx / BX, b = idx - a * BX;
            const unsigned char d = sT[a * L::BOXW + b + 3];
            unsigned char f = 0;
            if (d != 0) {
                const T* c = sU + (a + 3) * RW + (b + 6);
                const bool ty = trouble_cell(c, RW);
                f = (ty || (d == 1 && !trouble_cell(c, 1))) ? 1 : 0;
            }
            sPY[idx] = f;
        }
        __syncthreads();
    }

    // Phase 2: every x face and y face of the tile, once (one thread per
    // face; x and y faces share the call, with pointers and strides chosen
    // per face).
    {
        // Whole warps iterate together (the limiter packing in meg7_pair
        // needs all 32 lanes); a lane past the last face repeats it and
        // stores nothing.
        for (int w0 = tid & ~31; w0 < L::NF; w0 += NT) {
            const bool valid = w0 + (tid & 31) < L::NF;
            const int w = valid ? w0 + (tid & 31) : L::NF - 1;
            const bool xf = w < L::NHX;
            FaceIn<T> in;
            T inv_n, inv_t;
            int r = 0, f = 0, c = 0, w2 = 0;
            if (xf) {
                r = w / L::HXW;
                f = w - r * L::HXW;
                const int ry = r + 6, rx = f + 5;  // left cell of the face
                const T* u = sU + ry * RW + rx;
                in.u[0] = u;
                in.u[1] = u + NU;
                in.u[2] = u + 2 * NU;
                in.u[3] = u + 3 * NU;
                in.su = 1;
                const T* gx = sGX + (r + V) * L::GXW + (rx - 3);
                in.g[0] = gx;
                in.g[1] = gx + L::NGX;
                in.g[2] = gx + 2 * L::NGX;
                in.g[3] = gx + 3 * L::NGX;
                in.sg = 1;
                in.tr = sPX + r * L::PXW + (rx - 3);
                in.st = 1;
                const T* fx = sFX + r * L::FXW + (rx - 1);
                in.f[0] = fx;
                in.f[1] = fx + L::NFX;
                in.f[2] = fx + 2 * L::NFX;
                in.f[3] = fx + 3 * L::NFX;
                in.sf = 1;
                const T* ty = sGY + (ry - 3) * L::GYW + (rx - 6 + V);
                in.tun = ty + L::NGY;      // d u / d y (cons: d rho u / d y)
                in.tut = ty + 2 * L::NGY;  // d v / d y (cons: d rho v / d y)
                in.stq = 1;
                if constexpr (CONS) {
                    const T* qc = sQc + ry * RW + rx;
                    in.q[0] = qc;
                    in.q[1] = qc + NU;
                    in.q[2] = qc + 2 * NU;
                    in.q[3] = qc + 3 * NU;
                    in.tr0 = ty;
                }
                inv_n = inv_dx;
                inv_t = inv_dy;
            } else {
                w2 = w - L::NHX;
                f = w2 / BX;
                c = w2 - f * BX;
                const int ry = f + 5, rx = c + 6;  // lower cell of the face
                const T* u = sU + ry * RW + rx;
                in.u[0] = u;
                in.u[1] = u + 2 * NU;  // normal velocity v
                in.u[2] = u + NU;      // tangential velocity u
                in.u[3] = u + 3 * NU;
                in.su = RW;
                const T* gy = sGY + (ry - 3) * L::GYW + (rx - 6 + V);
                in.g[0] = gy;
                in.g[1] = gy + 2 * L::NGY;
                in.g[2] = gy + L::NGY;
                in.g[3] = gy + 3 * L::NGY;
                in.sg = L::GYW;
                in.tr = sPY + (ry - 3) * BX + c;
                in.st = BX;
                const T* fy = sFY + (ry - 1) * BX + c;
                in.f[0] = fy;
                in.f[1] = fy + 2 * L::NFY;  // rho v^2 + p
                in.f[2] = fy + L::NFY;      // rho u v
                in.f[3] = fy + 3 * L::NFY;
                in.sf = BX;
                const T* tx = sGX + (ry - 6 + V) * L::GXW + (rx - 3);
                in.tun = tx + 2 * L::NGX;  // d v / d x (cons: d rho v / d x)
                in.tut = tx + L::NGX;      // d u / d x (cons: d rho u / d x)
                in.stq = L::GXW;
                if constexpr (CONS) {
                    const T* qc = sQc + ry * RW + rx;
                    in.q[0] = qc;
                    in.q[1] = qc + 2 * NU;  // rho v
                    in.q[2] = qc + NU;      // rho u
                    in.q[3] = qc + 3 * NU;
                    in.tr0 = tx;
                }
                inv_n = inv_dy;
                inv_t = inv_dx;
            }
            T out[4];
            bool smooth;
            face_flux<T, VISC, ORDER, CONS>(in, ph, inv_n, inv_t, out, smooth);
            if (valid) {
                if (xf) {
#pragma unroll
                    for (int m = 0; m < 4; ++m) sHX[m * L::NHX + w] = out[m];
                    if (P.sigx) {
                        const int i = ty0 + r, jf = tx0 + f;
                        if (i < ny && jf <= nx) P.sigx[(long long)i * (nx + 1) + jf] = smooth ? 1 : 0;
                    }
                } else {
                    sHY[w2] = out[0];
                    sHY[L::NHY + w2] = out[2];
                    sHY[2 * L::NHY + w2] = out[1];
                    sHY[3 * L::NHY + w2] = out[3];
                    if (P.sigy) {
                        const int j = tx0 + c, iface = ty0 + f;
                        if (j < nx && iface <= ny) P.sigy[(long long)iface * nx + j] = smooth ? 1 : 0;
                    }
                }
            }
        }
    }
    __syncthreads();

    // Phase 3: residual (Eq. deriv) and the FP64 stage update (Eq. rk).
    const double dt = P.dt_ptr ? *P.dt_ptr : P.dt;
    const double cdt = P.cc * dt;
    T lam = T(0);  // max in T, widened once (the same value as widening each cell's)
    bool bad = false;
    for (int idx = tid; idx < BX * BY; idx += NT) {
        const int r = idx / BX, c = idx - r * BX;
        const int j = tx0 + c, i = ty0 + r;
        if (j >= nx || i >= ny) continue;
        double res[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const T dF = sHX[m * L::NHX + r * L::HXW + c + 1] - sHX[m * L::NHX + r * L::HXW + c];
            const T dG = sHY[m * L::NHY + (r + 1) * BX + c] - sHY[m * L::NHY + r * BX + c];
            res[m] = to_f64(-(rmul(dF, inv_dx) + rmul(dG, inv_dy)));
        }
        if (P.res) {
#pragma unroll
            for (int m = 0; m < 4; ++m) P.res[(long long)m * nx * ny + (long long)i * nx + j] = res[m];
        }
        if (P.qout) {
            const long long o = (long long)(i + kGhost) * pitch + (j + kGhost);
            double qv[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                double v = P.cb * P.q[o + m * plane] + cdt * res[m];
                if (P.ca != 0.0) v += P.ca * P.qn[o + m * plane];
                qv[m] = v;
            }
#pragma unroll
            for (int m = 0; m < 4; ++m) P.qout[o + m * plane] = qv[m];
            // Positivity in FP64: rho > 0 and p > 0 <=> 2 rho E > |rho u|^2
            // (the comparisons on the bits, off the FP64 pipe).
            const double e2 = 2.0 * qv[0] * qv[3] - (qv[1] * qv[1] + qv[2] * qv[2]);
            const bool ok = finite_bits(qv[0]) && finite_bits(qv[1]) && finite_bits(qv[2]) && finite_bits(qv[3]) &&
                            positive_bits(qv[0]) && positive_bits(e2);
            bad |= !ok;
            if (P.lam_out)  // Sec. 2.5 wavespeed of the new state
                lam = tmax_nan(lam, cell_wavespeed_t<T>(qv[0], qv[1], qv[2], qv[3], ph.gamma, ph.gm1, ph.mu,
                                                        inv_dx, inv_dy));
        }
    }
    if (P.qout) {
        if (__syncthreads_or(bad) && tid == 0) atomicOr(P.err, kErrNonPhysical);
    }
    if (P.lam_out) {
        __shared__ double red[NT / 32];
        const double lmax = warp_max(to_f64(lam));
        if ((tid & 31) == 0) red[tid >> 5] = lmax;
        __syncthreads();
        if (tid < 32) {
            double v = (tid < NT / 32) ? red[tid] : 0.0;
            v = warp_max(v);
            if (tid == 0) atomicMax(P.lam_out, (unsigned long long)__double_as_longlong(v));
        }
    }
    __syncthreads();
}

// One CTA per tile; the tile + halo is staged by a tensor copy described by
// tmap (the stage's input state, see encode_state_map). Each instance is
// held to the register budget of the CTAs per SM that its shared memory
// allows (FP64: 2, 1 for MEG7-cons; FP32: 3, 2 viscous or MEG7-cons): small
// source changes could otherwise push the allocation over the budget and cut
// the resident warps.
template <typename T, bool VISC, bool CONS, int LEARNED = 0>
constexpr int stage_min_blocks()
{
    return sizeof(T) == 8 ? (CONS ? 1 : 2) : ((VISC || CONS || LEARNED == 2) ? 2 : 3);
}

template <typename T, int BX, int BY, int NT, bool VISC, int LEARNED, int ORDER, bool CONS>
__global__ void __launch_bounds__(NT, stage_min_blocks<T, VISC, CONS, LEARNED>()) stage_kernel(const StageParams P, const __grid_constant__ CUtensorMap tmap)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    stage_tile<T, BX, BY, NT, VISC, LEARNED, ORDER, CONS, true>(P, blockIdx.x * BX, blockIdx.y * BY, smem_raw,
                                                                 &tmap);
}

template <typename T, int BX, int BY, int NT, bool VISC, int LEARNED = 0, int ORDER = 7, bool CONS = false>
cudaError_t launch_stage_t(const StageParams& p, cudaStream_t s)
{
    using L = TileLayout<BX, BY, VISC, CONS, sizeof(T) == 8>;
    constexpr size_t smem = L::template total_bytes<T, NT, LEARNED != 0>();
    static PerDevice<int> configured;  // the shared-memory limit is raised once per device
    auto kern = stage_kernel<T, BX, BY, NT, VISC, LEARNED, ORDER, CONS>;
    int ok = 0;
    cudaError_t e = configured.get(&ok, [&](int* v) {
        *v = 1;
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (e != cudaSuccess) return e;
    CUtensorMap map;
    e = encode_state_map(p.g, p.q, L::RW, L::RH, &map);
    if (e != cudaSuccess) return e;
    dim3 grid((p.g.nx + BX - 1) / BX, (p.g.ny + BY - 1) / BY);
    kern<<<grid, NT, smem, s>>>(p, map);
    return cudaGetLastError();
}

}  // namespace gbr
