// Region evaluation (the hot loop): for each region on the eval list, the
// nested Clenshaw-Curtis pair Q_N (coarse, N intervals per dimension) and Q_2N
// (fine, 2N intervals) of the bubble integrand, and err = |Q_N - Q_2N|
// (Sec. 3; Listing 3 evaluates the four children of a split this way).
//
// Integrand (Sec. 2, Eq. chi_ph / chi_pp after the Matsubara sum):
//   ph: f_l(k) f_m(k+q) F(e(k), e(k+q)),   pp: f_l(k) f_m(q-k) F(e(k), -e(q-k))
//   F(e1, e2) = [tanh(e1/2T) - tanh(e2/2T)] / (2 (e1 - e2))
// which equals [nF(e2) - nF(e1)]/(e1 - e2) for ph and, with e2 -> -e(q-k),
// [1 - nF(e1) - nF(e(q-k))]/(e1 + e(q-k)) for pp.  F is evaluated without
// cancellation from v = exp(-|x|), x = e/2T:
//   |d| <= 1/16, d = (e1 - e2)/2T:  F = (1/4T) sinhc(d) sech x1 sech x2
//                                      (tanh a - tanh b = sinh(a-b) sech a sech b)
//   same sign:      F = s (u2 - u1) / ((1+u1)(1+u2)(e1 - e2)),  u = v^2
//   opposite sign:  F = s (1 - u1 u2) / ((1+u1)(1+u2)(e1 - e2))
// with sech x = 2v/(1+u) and s the sign of x1.  One exp per energy and one
// division per node.
//
// Data reuse inside a region (tensor-product hoisting): the 2N+1 node
// abscissae per dimension are cos/sin rotations of the region centre, taken
// from sincospi of the exact dyadic centre and a per-level table of the node
// offsets, so a region costs 2 sincospi instead of 2(2N+1)^2 cos/sin.  The
// dispersion is affine in cos ky for fixed kx, e = A(kx) + B(kx) cos ky, and
// each form factor is X(kx)^T C Y(ky) with X = (1, cos kx, sin kx).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <type_traits>

#include "paid_internal.cuh"

namespace paid {

// rule variant v = (N - 4) / 2: N = 4 (5 x 5 coarse inside 9 x 9 fine), 6 (7 inside
// 13), and for the shared-partition kernel only 8, 10, 12 (13 inside 25)
__constant__ double c_wf[kRuleVariants][2 * kMaxRuleN + 1];   // fine CC weights on [-1, 1]
__constant__ double c_wc[kRuleVariants][kMaxRuleN + 1];       // coarse CC weights
__constant__ double c_t[kRuleVariants][2 * kMaxRuleN + 1];    // fine nodes t_i = cos(i pi / 2N)
__constant__ double c_co[kRuleVariants][kMaxLevel + 1][kMaxRuleN + 1];  // cos(pi 2^-L t_i), i <= N
__constant__ double c_so[kRuleVariants][kMaxLevel + 1][kMaxRuleN + 1];  // sin(pi 2^-L t_i)
__constant__ double c_ff[9][3][3];                // f_n = sum_ab C[a][b] X_a Y_b
__constant__ float c_wf32[2][2 * kMaxRuleNLow + 1];  // FP32 copies for the FP32 path
__constant__ float2 c_wfdf[2][2 * kMaxRuleNLow + 1]; // (hi, lo) pairs for the float-float path
__constant__ float2 c_wcdf[2][kMaxRuleNLow + 1];
__constant__ float2 c_exp2tab[64];                // 2^(j/64) as (hi, lo), j = 0..63
__constant__ float2 c_codf[2][kMaxLevel + 1][kMaxRuleNLow + 1];  // c_co / c_so as (hi, lo)
__constant__ float2 c_sodf[2][kMaxLevel + 1][kMaxRuleNLow + 1];
__constant__ float2 c_ffdf[9][3][3];              // c_ff as (hi, lo)
__constant__ float c_wc32[2][kMaxRuleNLow + 1];
__constant__ float c_ff32[9][3][3];
// the non-zero terms of c_ff: f_n = sum_{k < c_ffn[n]} c_ffc[n][k] X_a Y_b, a = c_ffa, b = c_ffb
__constant__ int c_ffn[9];
__constant__ int c_ffa[9][2];
__constant__ int c_ffb[9][2];
__constant__ double c_ffc[9][2];
__constant__ double c_exp2d[64];                  // 2^(j/64), j = 0..63 (FP64 exp of the group path)
// c_ffc[l][k1] c_ffc[m][k2] as float-float pairs (the FP32-pipe group kernel)
__constant__ float2 c_ffpair[9][2][9][2];

// Clenshaw-Curtis weights for n intervals (n even), from the cosine-series
// form of the rule: w_j = (c_j / n) (1 - sum_{k=1}^{n/2} b_k cos(2 k j pi/n)/(4k^2 - 1)).
static void cc_weights(int n, double* w)
{
    for (int j = 0; j <= n; ++j) {
        double acc = 1.0;
        for (int k = 1; k <= n / 2; ++k) {
            double bk = (2 * k == n) ? 1.0 : 2.0;
            acc -= bk * std::cos(2.0 * k * j * kPi / n) / (4.0 * k * k - 1.0);
        }
        w[j] = ((j == 0 || j == n) ? 1.0 : 2.0) / n * acc;
    }
}

static cudaError_t group_kernel_attributes();

cudaError_t init_rule_tables(int device)
{
    static bool done[64] = {false};
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (done[device]) return cudaSuccess;
    double wf[kRuleVariants][2 * kMaxRuleN + 1] = {}, wc[kRuleVariants][kMaxRuleN + 1] = {};
    double t[kRuleVariants][2 * kMaxRuleN + 1] = {};
    double co[kRuleVariants][kMaxLevel + 1][kMaxRuleN + 1] = {};
    double so[kRuleVariants][kMaxLevel + 1][kMaxRuleN + 1] = {};
    const int Ns[kRuleVariants] = {4, 6, 8, 10, 12};
    for (int v = 0; v < kRuleVariants; ++v) {
        int N = Ns[v];
        cc_weights(2 * N, wf[v]);
        cc_weights(N, wc[v]);
        for (int i = 0; i <= 2 * N; ++i) t[v][i] = std::cos(i * kPi / (2 * N));
        t[v][N] = 0.0;
        for (int L = 0; L <= kMaxLevel; ++L)
            for (int i = 0; i <= N; ++i) {
                double o = std::ldexp(kPi, -L) * t[v][i];   // half side pi 2^-L times t_i
                co[v][L][i] = std::cos(o);
                so[v][L][i] = std::sin(o);
            }
    }
    const double r2 = std::sqrt(2.0);
    double ff[9][3][3] = {};
    ff[0][0][0] = 1.0;                      // 1
    ff[1][1][0] = 1.0; ff[1][0][1] = 1.0;   // cx + cy
    ff[2][1][0] = 1.0; ff[2][0][1] = -1.0;  // cx - cy
    ff[3][2][0] = r2;                       // sqrt2 sx
    ff[4][0][2] = r2;                       // sqrt2 sy
    ff[5][1][1] = 2.0;                      // 2 cx cy
    ff[6][2][2] = 2.0;                      // 2 sx sy
    ff[7][2][1] = 2.0;                      // 2 sx cy
    ff[8][1][2] = 2.0;                      // 2 cx sy
    float wf32[2][2 * kMaxRuleNLow + 1], wc32[2][kMaxRuleNLow + 1], ff32[9][3][3];
    for (int v = 0; v < 2; ++v) {
        for (int i = 0; i < 2 * kMaxRuleNLow + 1; ++i) wf32[v][i] = float(wf[v][i]);
        for (int i = 0; i < kMaxRuleNLow + 1; ++i) wc32[v][i] = float(wc[v][i]);
    }
    for (int a = 0; a < 9; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) ff32[a][b][c] = float(ff[a][b][c]);
    float2 wfdf[2][2 * kMaxRuleNLow + 1], wcdf[2][kMaxRuleNLow + 1], e2t[64];
    auto split = [](double x) { float hi = float(x); return make_float2(hi, float(x - double(hi))); };
    for (int v = 0; v < 2; ++v) {
        for (int i = 0; i < 2 * kMaxRuleNLow + 1; ++i) wfdf[v][i] = split(wf[v][i]);
        for (int i = 0; i < kMaxRuleNLow + 1; ++i) wcdf[v][i] = split(wc[v][i]);
    }
    for (int j = 0; j < 64; ++j) e2t[j] = split(std::exp2(j / 64.0));
    float2 codf[2][kMaxLevel + 1][kMaxRuleNLow + 1], sodf[2][kMaxLevel + 1][kMaxRuleNLow + 1];
    float2 ffdf[9][3][3];
    for (int v = 0; v < 2; ++v)
        for (int L = 0; L <= kMaxLevel; ++L)
            for (int i = 0; i <= kMaxRuleNLow; ++i) {
                codf[v][L][i] = split(co[v][L][i]);
                sodf[v][L][i] = split(so[v][L][i]);
            }
    for (int a = 0; a < 9; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) ffdf[a][b][c] = split(ff[a][b][c]);
    cudaError_t e;
    if ((e = cudaMemcpyToSymbol(c_codf, codf, sizeof(codf))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_sodf, sodf, sizeof(sodf))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_ffdf, ffdf, sizeof(ffdf))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_wfdf, wfdf, sizeof(wfdf))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_wcdf, wcdf, sizeof(wcdf))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_exp2tab, e2t, sizeof(e2t))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_wf32, wf32, sizeof(wf32))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_wc32, wc32, sizeof(wc32))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_ff32, ff32, sizeof(ff32))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_wf, wf, sizeof(wf))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_wc, wc, sizeof(wc))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_t, t, sizeof(t))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_co, co, sizeof(co))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_so, so, sizeof(so))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_ff, ff, sizeof(ff))) != cudaSuccess) return e;
    int ffn[9] = {}, ffa[9][2] = {}, ffb[9][2] = {};
    double ffc[9][2] = {};
    for (int n = 0; n < 9; ++n)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                if (ff[n][a][b] != 0.0) {
                    ffa[n][ffn[n]] = a;
                    ffb[n][ffn[n]] = b;
                    ffc[n][ffn[n]] = ff[n][a][b];
                    ++ffn[n];
                }
    if ((e = cudaMemcpyToSymbol(c_ffn, ffn, sizeof(ffn))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_ffa, ffa, sizeof(ffa))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_ffb, ffb, sizeof(ffb))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_ffc, ffc, sizeof(ffc))) != cudaSuccess) return e;
    float2 ffpair[9][2][9][2] = {};
    for (int l = 0; l < 9; ++l)
        for (int k1 = 0; k1 < 2; ++k1)
            for (int m = 0; m < 9; ++m)
                for (int k2 = 0; k2 < 2; ++k2) ffpair[l][k1][m][k2] = split(ffc[l][k1] * ffc[m][k2]);
    if ((e = cudaMemcpyToSymbol(c_ffpair, ffpair, sizeof(ffpair))) != cudaSuccess) return e;
    double e2d[64];
    for (int j = 0; j < 64; ++j) e2d[j] = std::exp2(j / 64.0);
    if ((e = cudaMemcpyToSymbol(c_exp2d, e2d, sizeof(e2d))) != cudaSuccess) return e;
    if ((e = group_kernel_attributes()) != cudaSuccess) return e;
    done[device] = true;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// FP64 bubble kernel F(e1, e2) (see the file header), inv2T = 1/2T, inv4T = 1/4T.
__device__ __forceinline__ double bubble_F(double e1, double e2, double inv2T, double inv4T)
{
    const double diff = e1 - e2;
    const double d = diff * inv2T;
    const double x1 = e1 * inv2T, x2 = e2 * inv2T;
    const double v1 = exp(-fabs(x1)), v2 = exp(-fabs(x2));
    const double u1 = v1 * v1, u2 = v2 * v2;
    const double p = (1.0 + u1) * (1.0 + u2);
    const bool near = fabs(d) <= 0.0625;
    const bool neg1 = x1 < 0.0;
    const bool same = neg1 == (x2 < 0.0);
    double far = same ? (u2 - u1) : fma(-u1, u2, 1.0);
    far = neg1 ? -far : far;
    const double d2 = d * d;
    const double sinhc = fma(d2, fma(d2, fma(d2, fma(d2, 1.0 / 362880.0, 1.0 / 5040.0),
                                              1.0 / 120.0), 1.0 / 6.0), 1.0);
    const double nearv = (4.0 * inv4T) * (v1 * v2) * sinhc;
    const double num = near ? nearv : far;
    const double den = near ? p : p * diff;
    return num / den;
}

// Sum of the fine (w2) and coarse (w1) tensor rules over one region of a
// trigonometric-path kind (PH, PP, OVERLAP), in FP64.
template <int N, int KIND>
__device__ __forceinline__ void region_trig_fp64(int v, uint32_t L, uint32_t ix, uint32_t iy,
                                                 QTrig tq, int l, int m, const DevBatch& B,
                                                 Lattice lat, double& s2, double& s1)
{
    constexpr int NF = 2 * N + 1;
    const double inv2T = B.inv2T, inv4T = B.inv4T;
    // exact dyadic centre / pi: -1 + (2 ix + 1) 2^-L
    double sxc, cxc, syc, cyc;
    sincospi(fma(double(2 * ix + 1), ldexp(1.0, -int(L)), -1.0), &sxc, &cxc);
    sincospi(fma(double(2 * iy + 1), ldexp(1.0, -int(L)), -1.0), &syc, &cyc);

    double cy[NF], sy[NF], cy2[NF], sy2[NF];
#pragma unroll
    for (int j = 0; j < NF; ++j) {
        const int jj = j <= N ? j : 2 * N - j;
        const double co = c_co[v][L][jj];
        const double so = j <= N ? c_so[v][L][jj] : -c_so[v][L][jj];
        cy[j] = fma(cyc, co, -syc * so);
        sy[j] = fma(syc, co, cyc * so);
        if (KIND == PP) {   // q - k
            cy2[j] = fma(tq.cqy, cy[j], tq.sqy * sy[j]);
            sy2[j] = fma(tq.sqy, cy[j], -tq.cqy * sy[j]);
        } else {            // k + q
            cy2[j] = fma(cy[j], tq.cqy, -sy[j] * tq.sqy);
            sy2[j] = fma(sy[j], tq.cqy, cy[j] * tq.sqy);
        }
    }
    double Cl[3][3], Cm[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) { Cl[a][b] = c_ff[l][a][b]; Cm[a][b] = c_ff[m][a][b]; }

    const double tA = -2.0 * lat.t, tB = -4.0 * lat.tp;
    double fine = 0.0, coarse = 0.0;
#pragma unroll 1
    for (int i = 0; i < NF; ++i) {
        const int ii = i <= N ? i : 2 * N - i;
        const double co = c_co[v][L][ii];
        const double so = i <= N ? c_so[v][L][ii] : -c_so[v][L][ii];
        const double cx = fma(cxc, co, -sxc * so);
        const double sx = fma(sxc, co, cxc * so);
        double cx2, sx2;
        if (KIND == PP) { cx2 = fma(tq.cqx, cx, tq.sqx * sx); sx2 = fma(tq.sqx, cx, -tq.cqx * sx); }
        else            { cx2 = fma(cx, tq.cqx, -sx * tq.sqx); sx2 = fma(sx, tq.cqx, cx * tq.sqx); }
        // e = A + B cos ky along this row
        const double A1 = fma(tA, cx, -lat.mu), B1 = fma(tB, cx, tA);
        const double A2 = fma(tA, cx2, -lat.mu), B2 = fma(tB, cx2, tA);
        double ul[3], um[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            ul[b] = fma(Cl[2][b], sx, fma(Cl[1][b], cx, Cl[0][b]));
            um[b] = fma(Cm[2][b], sx2, fma(Cm[1][b], cx2, Cm[0][b]));
        }
        double rf = 0.0, rc = 0.0;
#pragma unroll
        for (int j = 0; j < NF; ++j) {
            double g;
            const double fl = fma(ul[2], sy[j], fma(ul[1], cy[j], ul[0]));
            const double fm = fma(um[2], sy2[j], fma(um[1], cy2[j], um[0]));
            if (KIND == OVERLAP) {
                g = fl * fm;
            } else {
                const double e1 = fma(B1, cy[j], A1);
                const double e2 = fma(B2, cy2[j], A2);
                g = fl * fm * bubble_F(e1, KIND == PP ? -e2 : e2, inv2T, inv4T);
            }
            rf = fma(c_wf[v][j], g, rf);
            if ((j & 1) == 0) rc = fma(c_wc[v][j >> 1], g, rc);
        }
        fine = fma(c_wf[v][i], rf, fine);
        if ((i & 1) == 0) coarse = fma(c_wc[v][i >> 1], rc, coarse);
    }
    s2 = fine;
    s1 = coarse;
}

// MONOMIAL test kind: (kx/pi)^l (ky/pi)^m; the rule is separable.
template <int N>
__device__ __forceinline__ void region_monomial(int v, uint32_t L, uint32_t ix, uint32_t iy,
                                                int a, int b, double& s2, double& s1)
{
    constexpr int NF = 2 * N + 1;
    const double hh = ldexp(1.0, -int(L));            // half side / pi
    const double xc = fma(double(2 * ix + 1), hh, -1.0), yc = fma(double(2 * iy + 1), hh, -1.0);
    double fx = 0.0, cxs = 0.0, fy = 0.0, cys = 0.0;
#pragma unroll
    for (int i = 0; i < NF; ++i) {
        const double px = pow(fma(hh, c_t[v][i], xc), double(a));
        const double py = pow(fma(hh, c_t[v][i], yc), double(b));
        fx = fma(c_wf[v][i], px, fx);
        fy = fma(c_wf[v][i], py, fy);
        if ((i & 1) == 0) {
            cxs = fma(c_wc[v][i >> 1], px, cxs);
            cys = fma(c_wc[v][i >> 1], py, cys);
        }
    }
    s2 = fx * fy;
    s1 = cxs * cys;
}

// ---------------------------------------------------------------------------
// FP32 evaluation (mixed precision).  What stays FP64: the region centre and
// node rotations, the reduced energies x = e/2T (1 DFMA each: the 1/2T factor
// is folded into the per-row coefficients) and their exact difference
// d = x1 - x2, because near the Fermi surface e is a small difference of O(1)
// terms and an FP32 energy would move x by ~1e-6 at T = 0.05; the region sums
// Q_N, Q_2N, their difference and all totals.  What runs in FP32: the
// kernel F from x1, x2, d (2 MUFU ex2 + one fast division per node), the form
// factors, and the sums of a row of nodes.
//
// Rounding noise.  Each node's FP32 value g = f_l f_m F carries independent
// rounding errors; their standard deviation, in units of 2^-24, is bounded by
//   s = kNoiseUlps |f_l f_m F|                 (ex2, products, division)
//     + 4 |F| (|f_l| + |f_m|)                   (form factors: sums of O(1) terms)
//     + |f_l f_m| dF                            (rounding x1, x2 to FP32)
// with dF = |F| (|x1| + |x2|) on the sinhc branch and
// dF = (sech^2 x1 |x1| + sech^2 x2 |x2|) / (2 |e1 - e2|) on the tanh branch
// (|dF/dx_i| |x_i| 2^-24 for F = (tanh x1 - tanh x2) / (2 (e1 - e2))).
// A region returns the rms noise of Q_N - Q_2N,
//   nse = 2^-24 (h/2)^2/(2pi)^2 sqrt(sum_ij (w_i w_j s_ij)^2 + sum_coarse (v_i v_j s_ij)^2),
// (w fine, v coarse weights).  The noise stays inside |Q_N - Q_2N| (it only
// makes the error estimate larger); an integral whose summed noise
// kNoiseSigmas * sum(nse) exceeds a quarter of its tolerance -- which no
// refinement can fix, since the sum does not shrink as regions split -- is
// re-evaluated at higher precision.
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// F(x1, x2) with x = e/2T, d = x1 - x2 (exact), twoT = 2T, inv4T = 1/4T, in FP32,
// and dF, the sensitivity of F to rounding x1, x2 (see the noise model above).
// |d| <= 1: (1/4T) sinhc(d) sech x1 sech x2 (series of sinhc to d^10);
// |d| > 1:  the same-sign / opposite-sign forms of the FP64 kernel.
__device__ __forceinline__ float bubble_F32(float x1, float x2, float d, float twoT, float inv4T,
                                            float& dF)
{
    const float L2E = 1.4426950408889634f;
    const float a1 = fabsf(x1), a2 = fabsf(x2);
    const float v1 = ex2_approx(-a1 * L2E), v2 = ex2_approx(-a2 * L2E);
    const float u1 = v1 * v1, u2 = v2 * v2;
    const float p1 = 1.0f + u1, p2 = 1.0f + u2;
    const float p = p1 * p2;
    const bool near = fabsf(d) <= 1.0f;
    const bool neg1 = x1 < 0.0f;
    const bool same = neg1 == (x2 < 0.0f);
    float far = same ? (u2 - u1) : fmaf(-u1, u2, 1.0f);
    far = neg1 ? -far : far;
    const float d2 = d * d;
    float sh = fmaf(d2, 1.0f / 39916800.0f, 1.0f / 362880.0f);
    sh = fmaf(d2, sh, 1.0f / 5040.0f);
    sh = fmaf(d2, sh, 1.0f / 120.0f);
    sh = fmaf(d2, sh, 1.0f / 6.0f);
    sh = fmaf(d2, sh, 1.0f);
    const float nearv = (4.0f * inv4T) * (v1 * v2) * sh;
    const float num = near ? nearv : far;
    const float ediff = twoT * d;   // e1 - e2
    const float den = near ? p : p * ediff;
    const float F = __fdividef(num, den);
    // sech^2 x = 4u / (1+u)^2
    const float s1 = __fdividef(4.0f * u1, p1 * p1), s2 = __fdividef(4.0f * u2, p2 * p2);
    dF = near ? fabsf(F) * (a1 + a2) : __fdividef(fmaf(s1, a1, s2 * a2), 2.0f * fabsf(ediff));
    return F;
}

template <int N, int KIND>
__device__ __forceinline__ void region_trig_fp32(int v, uint32_t L, uint32_t ix, uint32_t iy,
                                                 QTrig tq, int l, int m, const DevBatch& B,
                                                 Lattice lat, double& s2, double& s1, float& nz)
{
    constexpr int NF = 2 * N + 1;
    const double inv2T = B.inv2T;
    const float twoT = float(2.0 * B.T), inv4T = float(B.inv4T);
    double sxc, cxc, syc, cyc;
    sincospi(fma(double(2 * ix + 1), ldexp(1.0, -int(L)), -1.0), &sxc, &cxc);
    sincospi(fma(double(2 * iy + 1), ldexp(1.0, -int(L)), -1.0), &syc, &cyc);

    double cyd[NF], cy2d[NF];
    float cyf[NF], syf[NF], cy2f[NF], sy2f[NF];
#pragma unroll
    for (int j = 0; j < NF; ++j) {
        const int jj = j <= N ? j : 2 * N - j;
        const double co = c_co[v][L][jj];
        const double so = j <= N ? c_so[v][L][jj] : -c_so[v][L][jj];
        const double c = fma(cyc, co, -syc * so);
        const double sn = fma(syc, co, cyc * so);
        double c2, s2_;
        if (KIND == PP) { c2 = fma(tq.cqy, c, tq.sqy * sn); s2_ = fma(tq.sqy, c, -tq.cqy * sn); }
        else            { c2 = fma(c, tq.cqy, -sn * tq.sqy); s2_ = fma(sn, tq.cqy, c * tq.sqy); }
        cyd[j] = c;
        cy2d[j] = c2;
        cyf[j] = float(c);
        syf[j] = float(sn);
        cy2f[j] = float(c2);
        sy2f[j] = float(s2_);
    }
    float Cl[3][3], Cm[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) { Cl[a][b] = c_ff32[l][a][b]; Cm[a][b] = c_ff32[m][a][b]; }

    // x = e / 2T = A(kx) + B(kx) cos ky with A = (-2t cx - mu)/2T, B = (-2t - 4t' cx)/2T
    const double tA = -2.0 * lat.t * inv2T, tB = -4.0 * lat.tp * inv2T, mu = lat.mu * inv2T;
    double fine = 0.0, coarse = 0.0;
    float noise = 0.0f;
#pragma unroll 1
    for (int i = 0; i < NF; ++i) {
        const int ii = i <= N ? i : 2 * N - i;
        const double co = c_co[v][L][ii];
        const double so = i <= N ? c_so[v][L][ii] : -c_so[v][L][ii];
        const double cx = fma(cxc, co, -sxc * so);
        const double sx = fma(sxc, co, cxc * so);
        double cx2, sx2;
        if (KIND == PP) { cx2 = fma(tq.cqx, cx, tq.sqx * sx); sx2 = fma(tq.sqx, cx, -tq.cqx * sx); }
        else            { cx2 = fma(cx, tq.cqx, -sx * tq.sqx); sx2 = fma(sx, tq.cqx, cx * tq.sqx); }
        const double A1 = fma(tA, cx, -mu), B1 = fma(tB, cx, tA);
        const double A2 = fma(tA, cx2, -mu), B2 = fma(tB, cx2, tA);
        const float cxf = float(cx), sxf = float(sx), cx2f = float(cx2), sx2f = float(sx2);
        float ul[3], um[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            ul[b] = fmaf(Cl[2][b], sxf, fmaf(Cl[1][b], cxf, Cl[0][b]));
            um[b] = fmaf(Cm[2][b], sx2f, fmaf(Cm[1][b], cx2f, Cm[0][b]));
        }
        float rf = 0.0f, rc = 0.0f, rnf = 0.0f, rnc = 0.0f;
#pragma unroll
        for (int j = 0; j < NF; ++j) {
            const double x1 = fma(B1, cyd[j], A1);
            double x2 = fma(B2, cy2d[j], A2);
            if (KIND == PP) x2 = -x2;
            float dF;
            const float F = bubble_F32(float(x1), float(x2), float(x1 - x2), twoT, inv4T, dF);
            const float fl = fmaf(ul[2], syf[j], fmaf(ul[1], cyf[j], ul[0]));
            const float fm = fmaf(um[2], sy2f[j], fmaf(um[1], cy2f[j], um[0]));
            const float flm = fl * fm;
            const float g = flm * F;
            rf = fmaf(c_wf32[v][j], g, rf);
            if ((j & 1) == 0) rc = fmaf(c_wc32[v][j >> 1], g, rc);
            const float sg = fmaf(fabsf(flm), fmaf(kNoiseUlps, fabsf(F), dF),
                                  4.0f * fabsf(F) * (fabsf(fl) + fabsf(fm)));
            const float sf = c_wf32[v][j] * sg;
            rnf = fmaf(sf, sf, rnf);
            if ((j & 1) == 0) { const float sc = c_wc32[v][j >> 1] * sg; rnc = fmaf(sc, sc, rnc); }
        }
        fine = fma(c_wf[v][i], double(rf), fine);
        if ((i & 1) == 0) {
            coarse = fma(c_wc[v][i >> 1], double(rc), coarse);
            noise = fmaf(c_wc32[v][i >> 1] * c_wc32[v][i >> 1], rnc, noise);
        }
        noise = fmaf(c_wf32[v][i] * c_wf32[v][i], rnf, noise);
    }
    s2 = fine;
    s1 = coarse;
    nz = noise;
}

// ---------------------------------------------------------------------------
// Float-float ("df32") evaluation: every quantity is an unevaluated sum
// hi + lo of two FP32 numbers (about 48 significant bits), so the whole
// integrand runs on the FP32 pipe -- 64x the FP64 pipe on this GPU -- at
// close to FP64 accuracy.  Integrals whose FP32 rounding noise is too large
// for their tolerance (those that vanish by symmetry, mostly) are evaluated
// this way.  Building blocks, written from the published error-free
// transformations: Knuth's TwoSum, the FMA form of Dekker's TwoProduct, and
// the double-word add / multiply / divide of Hida, Li and Bailey's
// double-double arithmetic transposed to FP32 pairs.  Additions use the
// "sloppy" form (absolute error ~2^-48 of the operands), which is enough
// here: every sum is either of O(1) bounded terms or bounded away from
// cancellation (|d| > 1/8 on the tanh branch).
struct f2 {
    float hi, lo;
};

__device__ __forceinline__ f2 two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ f2 fast_two_sum(float a, float b)
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ f2 df_add(f2 a, f2 b)
{
    f2 s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ f2 df_add_f(f2 a, float b)
{
    f2 s = two_sum(a.hi, b);
    s.lo += a.lo;
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ f2 df_neg(f2 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ f2 df_mul(f2 a, f2 b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ f2 df_mul_f(f2 a, float b)
{
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// a / b: a first quotient from the approximate reciprocal, one correction
// from the exact residual a - q1 b.
__device__ __forceinline__ f2 df_div(f2 a, f2 b)
{
    const float r = rcp_approx(b.hi);
    const float q1 = a.hi * r;
    const f2 res = df_add(a, df_neg(df_mul_f(b, q1)));
    const float q2 = res.hi * r;
    return fast_two_sum(q1, q2);
}
__device__ __forceinline__ f2 df_from(double x)
{
    const float hi = float(x);
    return {hi, float(x - double(hi))};
}
__device__ __forceinline__ f2 df_c(float2 c) { return {c.x, c.y}; }

// exp(-a), a >= 0, in float-float (Tang's table-driven method): k = rint(64 a / ln 2),
// r = a - k ln2/64 with ln2/64 split in three parts so that k * C1 is exact
// (k < 2^14, C1 has 10 significant bits), e^-a = 2^(-k/64) e^-r with the
// table 2^(j/64) and a degree-5 Taylor polynomial of e^-r on |r| <= ln2/128
// (truncation below 4e-17).  Results below 2^-126 are flushed to zero.
__device__ __forceinline__ f2 df_exp_neg(f2 a, const float2* tab)
{
    if (a.hi > 87.0f) return {0.0f, 0.0f};
    const float C1 = 0.010833740234375f;          // 0x1.63p-7
    const float C2 = -3.3155381515825866e-06f;
    const float C3 = 2.572804640231345e-14f;
    // k = rint(64 a_hi / ln2) by the shift 1.5 * 2^23 (a_hi 64/ln2 < 2^13):
    // the low encoding bits of the sum are k
    const float kt = fmaf(a.hi, 92.33248138427734f, 12582912.0f);
    const float k = __fsub_rn(kt, 12582912.0f);
    const float t1 = fmaf(-k, C1, a.hi);          // exact (Sterbenz)
    f2 r = two_sum(t1, a.lo);
    const f2 kc2 = {k * C2, fmaf(k, C2, -k * C2)};
    r = df_add(r, df_neg(kc2));
    r = df_add_f(r, -k * C3);
    const f2 t = df_neg(r);                       // e^-a = 2^(-k/64) e^t
    float p = fmaf(t.hi, 1.0f / 120.0f, 1.0f / 24.0f);
    p = fmaf(t.hi, p, 1.0f / 6.0f);               // 1/6 + t/24 + t^2/120
    f2 P = df_add_f(df_mul_f(t, p), 0.5f);
    P = df_add_f(df_mul(t, P), 1.0f);
    P = df_add_f(df_mul(t, P), 1.0f);
    const int n = 0x4B400000 - __float_as_int(kt);   // -k
    const int m = n >> 6;                         // floor(n / 64)
    const int j = n & 63;
    f2 res = df_mul(P, df_c(tab[j]));
    if (m < -125) return {0.0f, 0.0f};
    const float sc = __int_as_float((m + 127) << 23);
    res.hi *= sc;
    res.lo *= sc;
    return res;
}

// F(x1, x2) = [tanh x1 - tanh x2] / (2 (e1 - e2)) in float-float, x = e / 2T,
// d = x1 - x2; |d| <= 1/8: (1/4T) sinhc(d) sech x1 sech x2; else the
// same-sign / opposite-sign forms of the FP64 kernel.
__device__ __forceinline__ f2 bubble_Fdf(f2 x1, f2 x2, f2 d, f2 twoT, f2 inv4T,
                                         const float2* tab)
{
    const bool neg1 = x1.hi < 0.0f, neg2 = x2.hi < 0.0f;
    const f2 a1 = neg1 ? df_neg(x1) : x1, a2 = neg2 ? df_neg(x2) : x2;
    const f2 v1 = df_exp_neg(a1, tab), v2 = df_exp_neg(a2, tab);
    const f2 u1 = df_mul(v1, v1), u2 = df_mul(v2, v2);
    const f2 p = df_mul(df_add_f(u1, 1.0f), df_add_f(u2, 1.0f));
    f2 num, den;
    if (fabsf(d.hi) <= 0.125f) {
        // sinhc(d) = 1 + d^2/6 + d^4/120 + d^6/5040 + d^8/362880 (+ < 3e-17 at |d| = 1/8)
        const f2 d2 = df_mul(d, d);
        const float q = fmaf(d2.hi, fmaf(d2.hi, 1.0f / 362880.0f, 1.0f / 5040.0f), 1.0f / 120.0f);
        f2 S = df_add(df_mul_f(d2, q), f2{0.1666666716337204f, -4.967053879312289e-09f});
        S = df_add_f(df_mul(d2, S), 1.0f);
        num = df_mul(df_mul(df_mul_f(inv4T, 4.0f), df_mul(v1, v2)), S);
        den = p;
    } else {
        num = (neg1 == neg2) ? df_add(u2, df_neg(u1)) : df_add_f(df_neg(df_mul(u1, u2)), 1.0f);
        if (neg1) num = df_neg(num);
        den = df_mul(p, df_mul(d, twoT));   // (e1 - e2) = 2T d
    }
    return df_div(num, den);
}

// Column values of a region: cos/sin of ky and of the shifted ky (4 x NF
// float-float numbers).  Kept in registers, or -- when ys is a shared-memory
// slice -- at ys[(f NF + j) kYsStride] (thread-minor, bank-conflict free),
// which frees 72 registers and lets more warps hide the latency of the
// float-float dependency chains.
constexpr int kYsStride = 128;   // threads per block of the float-float kernel

template <int NF>
struct YCols {
    float2* ys;                  // shared slice, or null for registers
    f2 r[4][NF];
    __device__ __forceinline__ void set(int f, int j, f2 v)
    {
        if (ys) ys[(f * NF + j) * kYsStride] = make_float2(v.hi, v.lo);
        else r[f][j] = v;
    }
    __device__ __forceinline__ f2 get(int f, int j) const
    {
        if (ys) { const float2 t = ys[(f * NF + j) * kYsStride]; return {t.x, t.y}; }
        return r[f][j];
    }
};

template <int N, int KIND, bool SMEM>
__device__ __forceinline__ void region_trig_df(int v, uint32_t L, uint32_t ix, uint32_t iy,
                                               QTrig tq, int l, int m, const DevBatch& B,
                                               Lattice lat, const float2* tab, float2* ys,
                                               double& s2, double& s1)
{
    constexpr int NF = 2 * N + 1;
    const double inv2T = B.inv2T;
    const f2 twoT = df_from(2.0 * B.T);
    const f2 inv4T = df_from(B.inv4T);
    // FP64 only for the exact dyadic centre; rotations, energies and form
    // factors below are float-float
    double sxc_, cxc_, syc_, cyc_;
    sincospi(fma(double(2 * ix + 1), ldexp(1.0, -int(L)), -1.0), &sxc_, &cxc_);
    sincospi(fma(double(2 * iy + 1), ldexp(1.0, -int(L)), -1.0), &syc_, &cyc_);
    const f2 cxc = df_from(cxc_), sxc = df_from(sxc_), cyc = df_from(cyc_), syc = df_from(syc_);
    const f2 cqx = df_from(tq.cqx), sqx = df_from(tq.sqx), cqy = df_from(tq.cqy), sqy = df_from(tq.sqy);

    YCols<NF> Y;
    Y.ys = SMEM ? ys : nullptr;
#pragma unroll
    for (int j = 0; j < NF; ++j) {
        const int jj = j <= N ? j : 2 * N - j;
        const f2 co = df_c(c_codf[v][L][jj]);
        const f2 so = j <= N ? df_c(c_sodf[v][L][jj]) : df_neg(df_c(c_sodf[v][L][jj]));
        const f2 c = df_add(df_mul(cyc, co), df_neg(df_mul(syc, so)));
        const f2 sn = df_add(df_mul(syc, co), df_mul(cyc, so));
        f2 c2, s2_;
        if (KIND == PP) {   // q - k
            c2 = df_add(df_mul(cqy, c), df_mul(sqy, sn));
            s2_ = df_add(df_mul(sqy, c), df_neg(df_mul(cqy, sn)));
        } else {            // k + q
            c2 = df_add(df_mul(c, cqy), df_neg(df_mul(sn, sqy)));
            s2_ = df_add(df_mul(sn, cqy), df_mul(c, sqy));
        }
        Y.set(0, j, c);
        Y.set(1, j, sn);
        Y.set(2, j, c2);
        Y.set(3, j, s2_);
    }
    // x = e / 2T = A(kx) + B(kx) cos ky, A = -(2t cx + mu)/2T, B = -(2t + 4t' cx)/2T
    const f2 tA = df_from(-2.0 * lat.t * inv2T), tB = df_from(-4.0 * lat.tp * inv2T);
    const f2 nmu = df_from(-lat.mu * inv2T);
    double fine = 0.0, coarse = 0.0;
#pragma unroll 1
    for (int i = 0; i < NF; ++i) {
        const int ii = i <= N ? i : 2 * N - i;
        const f2 co = df_c(c_codf[v][L][ii]);
        const f2 so = i <= N ? df_c(c_sodf[v][L][ii]) : df_neg(df_c(c_sodf[v][L][ii]));
        const f2 cx = df_add(df_mul(cxc, co), df_neg(df_mul(sxc, so)));
        const f2 sx = df_add(df_mul(sxc, co), df_mul(cxc, so));
        f2 cx2, sx2;
        if (KIND == PP) {
            cx2 = df_add(df_mul(cqx, cx), df_mul(sqx, sx));
            sx2 = df_add(df_mul(sqx, cx), df_neg(df_mul(cqx, sx)));
        } else {
            cx2 = df_add(df_mul(cx, cqx), df_neg(df_mul(sx, sqx)));
            sx2 = df_add(df_mul(sx, cqx), df_mul(cx, sqx));
        }
        const f2 A1 = df_add(df_mul(tA, cx), nmu), B1 = df_add(df_mul(tB, cx), tA);
        const f2 A2 = df_add(df_mul(tA, cx2), nmu), B2 = df_add(df_mul(tB, cx2), tA);
        f2 ul[3], um[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            ul[b] = df_add(df_add(df_mul(df_c(c_ffdf[l][1][b]), cx), df_mul(df_c(c_ffdf[l][2][b]), sx)),
                           df_c(c_ffdf[l][0][b]));
            um[b] = df_add(df_add(df_mul(df_c(c_ffdf[m][1][b]), cx2), df_mul(df_c(c_ffdf[m][2][b]), sx2)),
                           df_c(c_ffdf[m][0][b]));
        }
        f2 rf = {0.0f, 0.0f}, rc = {0.0f, 0.0f};
#pragma unroll
        for (int j = 0; j < NF; ++j) {
            const f2 cyj = Y.get(0, j), syj = Y.get(1, j), cy2j = Y.get(2, j), sy2j = Y.get(3, j);
            const f2 x1 = df_add(df_mul(B1, cyj), A1);
            f2 x2 = df_add(df_mul(B2, cy2j), A2);
            if (KIND == PP) x2 = df_neg(x2);
            const f2 F = bubble_Fdf(x1, x2, df_add(x1, df_neg(x2)), twoT, inv4T, tab);
            const f2 fl = df_add(df_add(df_mul(ul[1], cyj), df_mul(ul[2], syj)), ul[0]);
            const f2 fm = df_add(df_add(df_mul(um[1], cy2j), df_mul(um[2], sy2j)), um[0]);
            const f2 g = df_mul(df_mul(fl, fm), F);
            rf = df_add(rf, df_mul(df_c(c_wfdf[v][j]), g));
            if ((j & 1) == 0) rc = df_add(rc, df_mul(df_c(c_wcdf[v][j >> 1]), g));
        }
        fine = fma(c_wf[v][i], double(rf.hi) + double(rf.lo), fine);
        if ((i & 1) == 0) coarse = fma(c_wc[v][i >> 1], double(rc.hi) + double(rc.lo), coarse);
    }
    s2 = fine;
    s1 = coarse;
}

// PH / PP regions of integrals escalated to float-float (and not set to FP64).
__device__ __forceinline__ bool is_df_region(uint32_t mt)
{
    const int kind = meta_kind(mt);
    return meta_valid(mt) && (mt & kMetaDf32) != 0u && (mt & kMetaFp64) == 0u &&
           (kind == PH || kind == PP);
}

// Float-float evaluation kernel: one region per thread, the column values in
// a shared-memory slice per thread (N = 4) so that three 128-thread blocks fit
// per SM without spills.
template <int N>
__global__ void __launch_bounds__(kYsStride, N == 4 ? 3 : 1)
k_eval_df(Work w, Lattice lat)
{
    const int cur = w.ls->cur;
    const int64_t n_eval = w.ls->n_eval;
    constexpr bool SMEM = N == 4;
    constexpr int NF = 2 * N + 1;
    const int v = N == 4 ? 0 : 1;
    __shared__ float2 tab[64];
    __shared__ float2 ysm[SMEM ? 4 * NF * kYsStride : 1];
    if (threadIdx.x < 64) tab[threadIdx.x] = c_exp2tab[threadIdx.x];
    __syncthreads();
    float2* ys = SMEM ? ysm + threadIdx.x : nullptr;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    unsigned count = 0;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n_eval; t += stride) {
        const uint2 e = w.evl[t];
        const uint32_t pos = e.x, g = e.y;
        const uint32_t mt = w.meta[g];
        if (!is_df_region(mt)) continue;
        ++count;
        const uint64_t key = w.key[cur][pos];
        const DevBatch& B = w.batches[meta_batch(mt)];
        const uint32_t L = key_level(key), ix = key_ix(key), iy = key_iy(key);
        const QTrig tq = w.trig[g];
        const int l = meta_l(mt), m = meta_m(mt);
        double s2, s1;
        if (meta_kind(mt) == PH)
            region_trig_df<N, PH, SMEM>(v, L, ix, iy, tq, l, m, B, lat, tab, ys, s2, s1);
        else
            region_trig_df<N, PP, SMEM>(v, L, ix, iy, tq, l, m, B, lat, tab, ys, s2, s1);
        const double scale = ldexp(0.25, -2 * int(L));
        const double q2 = s2 * scale, q1 = s1 * scale;
        w.val[cur][pos] = q2;
        w.err[cur][pos] = fabs(q1 - q2);
        w.nse[cur][pos] = 0.0f;   // ~2^-44 relative: below every accepted tolerance
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) count += __shfl_xor_sync(0xffffffffu, count, o);
    if ((threadIdx.x & 31) == 0 && count) atomicAdd(&w.totals->df_regions, (unsigned long long)count);
}

// Mixed-precision evaluation: PH / PP regions use the FP32 path (regions of
// integrals escalated to float-float are left to k_eval_df); integrals set to
// FP64 and the test kinds use the FP64 path.
template <int N>
__global__ void __launch_bounds__(128) k_eval_fp32(Work w, Lattice lat)
{
    const int cur = w.ls->cur;
    const int64_t n_eval = w.ls->n_eval;
    const int v = N == 4 ? 0 : 1;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n_eval; t += stride) {
        const uint2 e = w.evl[t];
        const uint32_t pos = e.x, g = e.y;
        const uint32_t mt = w.meta[g];
        if (is_df_region(mt)) continue;   // evaluated by k_eval_df
        const uint64_t key = w.key[cur][pos];
        const DevBatch& B = w.batches[meta_batch(mt)];
        const uint32_t L = key_level(key), ix = key_ix(key), iy = key_iy(key);
        const int kind = meta_kind(mt);
        double s2 = NAN, s1 = NAN;
        float nz = 0.0f;
        if (meta_valid(mt)) {
            const QTrig tq = w.trig[g];
            const int l = meta_l(mt), m = meta_m(mt);
            const bool fp64 = (mt & kMetaFp64) != 0u;
            if (kind == PH && !fp64)
                region_trig_fp32<N, PH>(v, L, ix, iy, tq, l, m, B, lat, s2, s1, nz);
            else if (kind == PP && !fp64)
                region_trig_fp32<N, PP>(v, L, ix, iy, tq, l, m, B, lat, s2, s1, nz);
            else if (kind == PH)
                region_trig_fp64<N, PH>(v, L, ix, iy, tq, l, m, B, lat, s2, s1);
            else if (kind == PP)
                region_trig_fp64<N, PP>(v, L, ix, iy, tq, l, m, B, lat, s2, s1);
            else if (kind == OVERLAP)
                region_trig_fp64<N, OVERLAP>(v, L, ix, iy, tq, l, m, B, lat, s2, s1);
            else
                region_monomial<N>(v, L, ix, iy, l, m, s2, s1);
        }
        const double scale = ldexp(0.25, -2 * int(L));
        const double q2 = s2 * scale, q1 = s1 * scale;
        w.val[cur][pos] = q2;
        w.err[cur][pos] = fabs(q1 - q2);
        // nz = sum (w_i w_j s_ij)^2: rms noise 2^-24 scale sqrt(nz)
        w.nse[cur][pos] = float(sqrt(double(nz)) * scale * 5.9604644775390625e-8);
    }
}

template <int N>
__global__ void __launch_bounds__(128) k_eval_fp64(Work w, Lattice lat)
{
    const int cur = w.ls->cur;
    const int64_t n_eval = w.ls->n_eval;
    const int v = N == 4 ? 0 : 1;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n_eval; t += stride) {
        const uint2 e = w.evl[t];
        const uint32_t pos = e.x, g = e.y;
        const uint64_t key = w.key[cur][pos];
        const uint32_t mt = w.meta[g];
        const DevBatch& B = w.batches[meta_batch(mt)];
        const uint32_t L = key_level(key), ix = key_ix(key), iy = key_iy(key);
        const int kind = meta_kind(mt);
        double s2 = NAN, s1 = NAN;
        if (meta_valid(mt)) {
            const QTrig tq = w.trig[g];
            const int l = meta_l(mt), m = meta_m(mt);
            if (kind == PH)
                region_trig_fp64<N, PH>(v, L, ix, iy, tq, l, m, B, lat, s2, s1);
            else if (kind == PP)
                region_trig_fp64<N, PP>(v, L, ix, iy, tq, l, m, B, lat, s2, s1);
            else if (kind == OVERLAP)
                region_trig_fp64<N, OVERLAP>(v, L, ix, iy, tq, l, m, B, lat, s2, s1);
            else
                region_monomial<N>(v, L, ix, iy, l, m, s2, s1);
        }
        // (h/2)^2 / (2 pi)^2 with h = 2 pi 2^-L:  2^-2L / 4
        const double scale = ldexp(0.25, -2 * int(L));
        const double q2 = s2 * scale, q1 = s1 * scale;
        w.val[cur][pos] = q2;
        w.err[cur][pos] = fabs(q1 - q2);
        w.nse[cur][pos] = 0.0f;
    }
}

// ---------------------------------------------------------------------------
// FP64 exp and division of the shared-partition kernel.
//
// exp(-a), a >= 0: P. T. P. Tang's table-driven method (ACM TOMS 15, 1989):
// -a = n ln2/64 + r with n = round(-a 64/ln2) = 64 m + j, 0 <= j < 64, so
// exp(-a) = 2^m 2^(j/64) exp(r), |r| <= ln2/128.  r comes from a two-constant
// Cody-Waite reduction (L1 = ln2/64 to 32 significant bits, so n L1 is exact
// for |n| < 2^21; L2 = ln2/64 - L1), exp(r) from its degree-5 Taylor
// polynomial (truncation r^6/720 < 2^-54 on that interval) and 2^(j/64) from a
// 64-entry table; 2^m enters as an integer add to the exponent field.  Results
// below 2^-1022 flush to zero; NaN propagates.
__device__ __forceinline__ double exp_neg(double a, const double* tab)
{
    a = a > 800.0 ? 800.0 : a;
    const double n = rint(a * -92.33248261689366);
    double r = fma(n, -0x1.62e42ffp-7, -a);
    r = fma(n, 0x1.718432a1b0e26p-41, r);
    double p = fma(r, 1.0 / 120.0, 1.0 / 24.0);
    p = fma(r, p, 1.0 / 6.0);
    p = fma(r, p, 0.5);
    p = fma(r, p, 1.0);
    p = fma(r, p, 1.0);
    const int ni = int(n);
    const int m = ni >> 6;          // floor(n / 64)
    const int j = ni & 63;
    const double y = tab[j] * p;    // in [0.99, 2.02]: exponent field 1022 ... 1024
    const long long b = __double_as_longlong(y) + ((long long)m << 52);
    if (y != y) return y;           // NaN in, NaN out (the integer n of a NaN is arbitrary)
    return (m >= -1022 && (b >> 52) > 0) ? __longlong_as_double(b) : 0.0;
}

// num / den for a normal, non-zero den: the approximate FP64 reciprocal of
// the PTX ISA (rcp.approx.ftz.f64) refined by two Newton-Raphson steps
// y <- y + y (1 - den y), then one residual correction of the quotient
// q <- q + (num - den q) y.
__device__ __forceinline__ double div_nr(double num, double den)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(den));
    double e = fma(-den, y, 1.0);
    y = fma(y, e, y);
    e = fma(-den, y, 1.0);
    y = fma(y, e, y);
    const double q = num * y;
    return fma(fma(-den, q, num), y, q);
}

// 2T F from the reduced energies x1 = e1/2T, x2 = e2/2T (the group kernel
// folds 1/2T into its row coefficients and its region Jacobian): with
// d = x1 - x2 = (e1 - e2)/2T,
//   near (|d| <= 1/16):  2T F = v1 v2 (2 sinhc d) / ((1+u1)(1+u2))
//   far:                 2T F = s [u2 - u1 | 1 - u1 u2] / ((1+u1)(1+u2) d)
// (the same branches and identities as bubble_F, one factor 2T throughout).
__device__ __forceinline__ double bubble_F2T(double x1, double x2, const double* tab)
{
    const double d = x1 - x2;
    const double v1 = exp_neg(fabs(x1), tab), v2 = exp_neg(fabs(x2), tab);
    const double u1 = v1 * v1, u2 = v2 * v2;
    const double p = (1.0 + u1) * (1.0 + u2);
    const bool near = fabs(d) <= 0.0625;
    const bool neg1 = x1 < 0.0;
    const bool same = neg1 == (x2 < 0.0);
    double far = same ? (u2 - u1) : fma(-u1, u2, 1.0);
    far = neg1 ? -far : far;
    double num = far, den = p * d;
    // the near branch is needed only in the thin band |e(k) - e(k')| <= 2T/16
    // (all of the zone only near q = 0): a warp none of whose lanes is near
    // skips the series
    if (__any_sync(__activemask(), near)) {
        const double d2 = d * d;
        const double sinhc2 = fma(d2, fma(d2, fma(d2, fma(d2, 2.0 / 362880.0, 2.0 / 5040.0),
                                                   2.0 / 120.0), 2.0 / 6.0), 2.0);
        if (near) {
            num = (v1 * v2) * sinhc2;
            den = p;
        }
    }
    return div_nr(num, den);
}

// Omega derivative of the frequency integrals of the flow kinds (Sec. 2,
// regulator theta(k0) = k0^2 / (k0^2 + Omega^2), T = 0, measure dk0 / 2pi):
// the divided difference of Hdot(e) = e (3|e| + W) / (4 (|e| + W)^3) at
// (e1, e2) for ph and minus that at (e1, -e2) for pp.  With u = |e| + W:
// energies of one sign (Hdot odd and smooth there):
//   (-3 P^2 + 5 W S P - 2 W^2 (S^2 - P)) / (4 P^3),  P = u1 u2, S = u1 + u2
// (the exact divided difference of (3/u - 5W/u^2 + 2W^2/u^3) / 4);
// opposite signs (no cancellation):
//   (e1 (3|e1| + W) u2^3 - e2 (3|e2| + W) u1^3) / (4 u1^3 u2^3 (e1 - e2)).
__device__ __forceinline__ double flow_Fdot(double e1, double e2, double W, bool pp)
{
    if (pp) e2 = -e2;
    const double a1 = fabs(e1), a2 = fabs(e2);
    const double u1 = a1 + W, u2 = a2 + W;
    const double P = u1 * u2, S = u1 + u2;
    const bool same = (e1 >= 0.0) == (e2 >= 0.0);
    const double u13 = u1 * u1 * u1, u23 = u2 * u2 * u2;
    const double num_s = fma(-3.0 * P, P, W * fma(5.0 * S, P, -2.0 * W * fma(S, S, -P)));
    const double num_o = fma(e1 * fma(3.0, a1, W), u23, -e2 * fma(3.0, a2, W) * u13);
    const double num = same ? num_s : num_o;
    const double den = same ? 4.0 * P * P * P : 4.0 * u13 * u23 * (e1 - e2);
    const double D = div_nr(num, den);
    return pp ? -D : D;
}

// ---------------------------------------------------------------------------
// FP32-pipe evaluation of the shared-partition kernel (options.eval_fp32 with
// group_mode).  The kernel F and the row sums run in float-float on the FP32
// pipe (64x the FP64 pipe on this GPU); the moments, the pair values, their
// errors and every total stay FP64.  A float-float number is an unevaluated
// sum hi + lo of two FP32 numbers (about 48 significant bits).  The building
// blocks are the published error-free transformations: Knuth's TwoSum,
// Dekker's FastTwoSum (|a| >= |b|) and the FMA form of TwoProduct, combined as
// in double-word arithmetic.  Every product whose rounded value enters a
// TwoSum is written with __fmul_rn, which the compiler never contracts into
// an FMA, so that each transformation stays exact.
__device__ __forceinline__ f2 ff_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ f2 ff_fast(float a, float b)   // |a| >= |b| (or a = 0)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ f2 ff_from(double x)
{
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - double(h))};
}
__device__ __forceinline__ double ff_to(f2 a) { return double(a.hi) + double(a.lo); }
__device__ __forceinline__ f2 ff_neg(f2 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ f2 ff_add(f2 a, f2 b)
{
    const f2 s = ff_two_sum(a.hi, b.hi);
    return ff_fast(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ f2 ff_sub(f2 a, f2 b) { return ff_add(a, ff_neg(b)); }
// 1 + u for 0 <= u <= 1
__device__ __forceinline__ f2 ff_one_plus(f2 u)
{
    const f2 s = ff_fast(1.0f, u.hi);
    return ff_fast(s.hi, __fadd_rn(s.lo, u.lo));
}
__device__ __forceinline__ f2 ff_mul(f2 a, f2 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return ff_fast(p, e);
}
__device__ __forceinline__ f2 ff_sqr(f2 a)
{
    const float p = __fmul_rn(a.hi, a.hi);
    float e = fmaf(a.hi, a.hi, -p);
    e = fmaf(a.hi + a.hi, a.lo, e);
    return ff_fast(p, e);
}
// a b + c, normalised
__device__ __forceinline__ f2 ff_fma(f2 a, f2 b, f2 c)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const f2 s = ff_two_sum(c.hi, p);
    return ff_fast(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}
// c += a b with c an accumulator left unnormalised: hi takes the rounded
// running sum, lo every rounding error (exact TwoSum and TwoProduct errors and
// the cross terms), so lo stays within a few ulp of hi over a row of nodes;
// ff_fast(hi, lo) normalises at the end.
__device__ __forceinline__ void ff_acc(f2 a, f2 b, f2& c)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float s = __fadd_rn(c.hi, p);
    const float bb = __fsub_rn(s, c.hi);
    const float t = __fadd_rn(__fsub_rn(c.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    c.hi = s;
    c.lo = __fadd_rn(c.lo, __fadd_rn(t, e));
}
// a / b, b normal and non-zero: q1 = a_hi rcp(b_hi), one correction from the
// residual a - b q1 (its leading part a_hi - b_hi q1 is exact, Sterbenz).
__device__ __forceinline__ f2 ff_div(f2 a, f2 b)
{
    const float r = rcp_approx(b.hi);
    const float q1 = __fmul_rn(a.hi, r);
    const float p = __fmul_rn(b.hi, q1);
    const float e = fmaf(b.hi, q1, -p);
    float res = __fsub_rn(__fsub_rn(a.hi, p), e);
    res = fmaf(-b.lo, q1, res);
    res = __fadd_rn(res, a.lo);
    return ff_fast(q1, __fmul_rn(res, r));
}

// exp(-a) for a float-float a >= 0 (Tang's table-driven method, as exp_neg):
// a = k ln2/64 + r, k = rint(64 a / ln2), e^-a = 2^(-k/64) e^-r.  ln2/64 is
// split as C1 + C2 + C3 with C1 of 9 significant bits, so k C1 is exact for
// k < 2^15 and a_hi - k C1 is exact (Sterbenz); r is then formed in
// float-float.  e^t (t = -r, |t| <= 0.0055) = 1 + t + t^2/2 + t^3 (1/6 + t/24
// + t^2/120): the first three terms in float-float, the rest (< 3e-8) in FP32
// (error < 4e-15); truncation t^6/720 < 4e-17.  2^(j/64) comes from a
// float-float table and 2^m (m >= -73) scales both parts exactly.  a >= 50
// gives 0 (e^-50 < 2e-22: the kernel F only uses v^2 and products of v there,
// which flush to zero in FP32).
__device__ __forceinline__ f2 ff_exp_neg(f2 a, const float2* tab)
{
    if (!(a.hi < 50.0f)) return {a.hi != a.hi ? a.hi : 0.0f, 0.0f};
    const float C1 = 0.010833740234375f;          // 0x1.63p-7
    const float C2 = -3.3155381515825866e-06f;
    const float C3 = 2.572804640231345e-14f;
    // k = rint(64 a_hi / ln2) by the shift 1.5 * 2^23: the sum lies in
    // [2^23, 2^24), where the float grid is the integers, so its low encoding
    // bits are k (two FP32-pipe instructions in place of a float rounding and
    // a float-to-integer conversion)
    const float kt = fmaf(a.hi, 92.33248138427734f, 12582912.0f);
    const float k = __fsub_rn(kt, 12582912.0f);
    const float t1 = fmaf(-k, C1, a.hi);          // exact
    const f2 s1 = ff_two_sum(t1, a.lo);
    const float p2 = __fmul_rn(k, C2);
    const float e2 = fmaf(k, C2, -p2);
    const f2 s2 = ff_two_sum(s1.hi, -p2);
    float lo = __fadd_rn(s2.lo, s1.lo);
    lo = __fsub_rn(lo, e2);
    lo = fmaf(-k, C3, lo);
    const f2 r = ff_fast(s2.hi, lo);
    const float th = -r.hi, tl = -r.lo;           // t = -r
    const float h = __fmul_rn(th, th);
    const float hl = fmaf(th, th, -h);            // th^2 = h + hl
    float q = fmaf(th, 1.0f / 120.0f, 1.0f / 24.0f);
    q = fmaf(th, q, 1.0f / 6.0f);
    const float c = __fmul_rn(__fmul_rn(h, th), q);
    const f2 S = ff_fast(th, 0.5f * h);           // t + t^2/2, leading parts
    float sl = __fadd_rn(S.lo, tl);
    sl = fmaf(0.5f, hl, sl);
    sl = fmaf(th, tl, sl);
    sl = __fadd_rn(sl, c);
    const f2 P0 = ff_fast(1.0f, S.hi);
    const f2 P = ff_fast(P0.hi, __fadd_rn(P0.lo, sl));
    const int n = 0x4B400000 - __float_as_int(kt);   // -k
    const int m = n >> 6;                         // floor(n / 64)
    const int j = n & 63;
    const float2 tj = tab[j];
    const f2 y = ff_mul(P, f2{tj.x, tj.y});
    const float sc = __int_as_float((m + 127) << 23);
    return {__fmul_rn(y.hi, sc), __fmul_rn(y.lo, sc)};
}

// 2T F(x1, x2) in float-float from the reduced energies (x = e/2T, the same
// branches and identities as bubble_F2T): d = x1 - x2,
//   near (|d| <= 1/16):  v1 v2 (2 sinhc d) / ((1+u1)(1+u2))
//   far:                 s [u2 - u1 | 1 - u1 u2] / ((1+u1)(1+u2) d)
// 2 sinhc d = 2 + d^2/3 + d^4/60 + d^6/2520 + d^8/181440 (next term < 5e-20
// at |d| = 1/16), the d^2/3 term in float-float.
__device__ __forceinline__ f2 bubble_F2T_ff(f2 x1, f2 x2, const float2* tab)
{
    const f2 d = ff_sub(x1, x2);
    const bool neg1 = x1.hi < 0.0f, neg2 = x2.hi < 0.0f;
    const f2 v1 = ff_exp_neg(neg1 ? ff_neg(x1) : x1, tab);
    const f2 v2 = ff_exp_neg(neg2 ? ff_neg(x2) : x2, tab);
    const f2 u1 = ff_sqr(v1), u2 = ff_sqr(v2);
    const f2 p = ff_mul(ff_one_plus(u1), ff_one_plus(u2));
    const bool same = neg1 == neg2;
    const f2 u12 = ff_mul(u1, u2);
    f2 num = ff_sub(same ? u2 : f2{1.0f, 0.0f}, same ? u1 : u12);
    if (neg1) num = ff_neg(num);
    f2 den = ff_mul(p, d);
    const bool near = fabsf(d.hi) <= 0.0625f;
    if (__any_sync(__activemask(), near)) {
        const f2 d2 = ff_sqr(d);
        const float g = d2.hi;
        const float tail = __fmul_rn(__fmul_rn(g, g),
                                     fmaf(g, fmaf(g, 1.0f / 181440.0f, 1.0f / 2520.0f), 1.0f / 60.0f));
        const f2 third = ff_mul(d2, f2{0.3333333432674408f, -9.934107758624577e-09f});
        const f2 S0 = ff_fast(2.0f, third.hi);    // 2 > d^2/3: exact
        const f2 S = ff_fast(S0.hi, __fadd_rn(S0.lo, __fadd_rn(third.lo, tail)));
        if (near) {
            num = ff_mul(ff_mul(v1, v2), S);
            den = p;
        }
    }
    return ff_div(num, den);
}

// Omega derivative of the flow kinds' frequency integrals in float-float (the
// same formulas as flow_Fdot; e1, e2 energies, W = Omega as float-float).
__device__ __forceinline__ f2 flow_Fdot_ff(f2 e1, f2 e2, f2 W, bool pp)
{
    if (pp) e2 = ff_neg(e2);
    const bool n1 = e1.hi < 0.0f, n2 = e2.hi < 0.0f;
    const f2 a1 = n1 ? ff_neg(e1) : e1, a2 = n2 ? ff_neg(e2) : e2;
    const f2 u1 = ff_add(a1, W), u2 = ff_add(a2, W);
    const f2 P = ff_mul(u1, u2), S = ff_add(u1, u2);
    f2 num, den;
    if (n1 == n2) {
        // -3 P^2 + W (5 S P - 2 W (S^2 - P))
        const f2 inner = ff_sub(ff_mul(ff_mul(f2{5.0f, 0.0f}, S), P),
                                ff_mul(ff_mul(f2{2.0f, 0.0f}, W), ff_sub(ff_sqr(S), P)));
        num = ff_sub(ff_mul(W, inner), ff_mul(f2{3.0f, 0.0f}, ff_sqr(P)));
        den = ff_mul(f2{4.0f, 0.0f}, ff_mul(P, ff_sqr(P)));
    } else {
        const f2 u13 = ff_mul(u1, ff_sqr(u1)), u23 = ff_mul(u2, ff_sqr(u2));
        const f2 g1 = ff_mul(e1, ff_add(ff_mul(f2{3.0f, 0.0f}, a1), W));
        const f2 g2 = ff_mul(e2, ff_add(ff_mul(f2{3.0f, 0.0f}, a2), W));
        num = ff_sub(ff_mul(g1, u23), ff_mul(g2, u13));
        den = ff_mul(ff_mul(f2{4.0f, 0.0f}, ff_mul(u13, u23)), ff_sub(e1, e2));
    }
    const f2 D = ff_div(num, den);
    return pp ? ff_neg(D) : D;
}

// Diagnostics for paid_check_math: which = 0: exp_neg(x), 1: div_nr(x, y),
// 2: ff_exp_neg(x) (x rounded to float-float), 3: bubble_F2T_ff(x, y),
// 4: bubble_F2T(x, y) (FP64), 5: flow_Fdot_ff(x, y) with Omega = 0.1 (ph),
// 6: flow_Fdot(x, y) with Omega = 0.1 (ph).
__global__ void k_check_math(int which, int64_t n, const double* x, const double* y, double* out)
{
    __shared__ double tab[64];
    __shared__ float2 tabf[64];
    if (threadIdx.x < 64) {
        tab[threadIdx.x] = c_exp2d[threadIdx.x];
        const f2 a = ff_from(c_exp2d[threadIdx.x]);
        tabf[threadIdx.x] = make_float2(a.hi, a.lo);
    }
    __syncthreads();
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    switch (which) {
    case 0: out[i] = exp_neg(x[i], tab); break;
    case 1: out[i] = div_nr(x[i], y[i]); break;
    case 2: out[i] = ff_to(ff_exp_neg(ff_from(x[i]), tabf)); break;
    case 3: out[i] = ff_to(bubble_F2T_ff(ff_from(x[i]), ff_from(y[i]), tabf)); break;
    case 4: out[i] = bubble_F2T(x[i], y[i], tab); break;
    case 5: out[i] = ff_to(flow_Fdot_ff(ff_from(x[i]), ff_from(y[i]), ff_from(0.1), false)); break;
    default: out[i] = flow_Fdot(x[i], y[i], 0.1, false); break;
    }
}

cudaError_t launch_check_math(int which, int64_t n, const double* x, const double* y, double* out,
                              cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_check_math<<<int((n + 255) / 256), 256, 0, s>>>(which, n, x, y, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Shared-partition (group) evaluation: one region of a (kind, q) group gives
// Q_N and Q_2N of every (l, m) pair of the group's batch at once.  With
// g = (1, cos, sin) every form factor is f_n(k) = sum C_n[a][b] g_a(kx) g_b(ky),
// so with k' = k + q (ph) or q - k (pp)
//   f_l(k) f_m(k') = sum C_l[a][b] C_m[c][d] X_ac(kx) Y_bd(ky),
//   X_ac = g_a(kx) g_c(kx'),   Y_bd = g_b(ky) g_d(ky'),
// and the rule applied to every pair needs only the 81 moments
//   M[ac][bd] = sum_i wx_i X_ac(x_i) R_i[bd],   R_i[bd] = sum_j wy_j F_ij Y_bd(y_j)
// and their coarse-rule counterparts: the kernel F once per node, 81 NF FMA
// (fine) + 81 (N+1) (coarse) for the moments, at most 4 terms per pair.
// Block: NF = 2N+1 threads per region (thread i owns fine row i, and column
// i for the shared column data, and moment cells i, i + NF, ...),
// GroupShape<N>::R regions per block.
template <int N> struct GroupShape;
template <> struct GroupShape<4> { static constexpr int R = 14; };   // 126 threads
template <> struct GroupShape<6> { static constexpr int R = 9; };    // 117 threads
template <> struct GroupShape<8> { static constexpr int R = 7; };    // 119 threads
template <> struct GroupShape<10> { static constexpr int R = 6; };   // 126 threads
template <> struct GroupShape<12> { static constexpr int R = 5; };   // 125 threads

template <int N>
struct GroupSmem {
    static constexpr int NF = 2 * N + 1, R = GroupShape<N>::R;
    double X[R][NF][9];      // X_ac at the fine rows
    double Y[R][NF][9];      // Y_bd at the fine columns
    double CY[R][NF][2];     // cos ky, cos ky' at the fine columns
    double Rf[R][NF][9];     // fine row sums R_i[bd]
    double Rc[R][N + 1][9];  // coarse row sums (even rows)
    double Mf[R][9][9];      // fine moments
    double Mc[R][9][9];      // coarse moments
    double C[R][4];          // sin, cos of the region centre (x, y) times pi
    double tab[64];          // 2^(j/64)
};

template <int N>
__global__ void __launch_bounds__(GroupShape<N>::R * (2 * N + 1))
k_eval_group(Work w, Lattice lat, double* rule_q2, double* rule_d)
{
    constexpr int NF = 2 * N + 1, R = GroupShape<N>::R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GroupSmem<N>& S = *reinterpret_cast<GroupSmem<N>*>(smem_raw);
    const int v = rule_variant(N);
    const int cur = w.ls->cur;
    const int64_t n_eval = w.ls->n_eval;
    const int rho = threadIdx.x / NF, i = threadIdx.x % NF;
    const double tA = -2.0 * lat.t, tB = -4.0 * lat.tp;
    if (threadIdx.x < 64) S.tab[threadIdx.x] = c_exp2d[threadIdx.x];
    for (int64_t chunk = blockIdx.x; chunk * R < n_eval; chunk += gridDim.x) {
        const int64_t t = chunk * R + rho;
        const bool live = t < n_eval;
        uint32_t pos = 0, g = 0, L = 0;
        int kind = PH, P = 0;
        const DevBatch* B = nullptr;
        double A1 = 0.0, B1 = 0.0, A2 = 0.0, B2 = 0.0;
        uint64_t key = 0;
        if (live) {
            const uint2 e = w.evl[t];
            pos = e.x;
            g = e.y;
            key = w.key[cur][pos];
            L = key_level(key);
            if (i < 2) {   // the exact dyadic centre / pi: -1 + (2 ix + 1) 2^-L, x then y
                const uint32_t ic = i == 0 ? key_ix(key) : key_iy(key);
                sincospi(fma(double(2 * ic + 1), ldexp(1.0, -int(L)), -1.0), &S.C[rho][2 * i],
                         &S.C[rho][2 * i + 1]);
            }
        }
        __syncthreads();
        if (live) {
            const uint32_t mt = w.meta[g];
            B = &w.batches[meta_batch(mt)];
            kind = meta_kind(mt);
            P = B->npairs;
            const QTrig tq = w.trig[g];     // flow kinds: rotation by q/2
            const bool pp = kind == PP, flow = is_flow(kind);
            const double sxc = S.C[rho][0], cxc = S.C[rho][1];
            const double syc = S.C[rho][2], cyc = S.C[rho][3];
            const int ii = i <= N ? i : 2 * N - i;
            const double co = c_co[v][L][ii];
            const double so = i <= N ? c_so[v][L][ii] : -c_so[v][L][ii];
            // row i (x) and column i (y) of the fine grid, and the shifted k'
            const double cx = fma(cxc, co, -sxc * so), sx = fma(sxc, co, cxc * so);
            const double cy = fma(cyc, co, -syc * so), sy = fma(syc, co, cyc * so);
            const double cx2 = pp ? fma(tq.cqx, cx, tq.sqx * sx) : fma(cx, tq.cqx, -sx * tq.sqx);
            const double sx2 = pp ? fma(tq.sqx, cx, -tq.cqx * sx) : fma(sx, tq.cqx, cx * tq.sqx);
            const double cy2 = pp ? fma(tq.cqy, cy, tq.sqy * sy) : fma(cy, tq.cqy, -sy * tq.sqy);
            const double sy2 = pp ? fma(tq.sqy, cy, -tq.cqy * sy) : fma(sy, tq.cqy, cy * tq.sqy);
            // flow kinds: both form factors at k (symmetric routing)
            const double gx[3] = {1.0, cx, sx};
            const double gx2[3] = {1.0, flow ? cx : cx2, flow ? sx : sx2};
            const double gy[3] = {1.0, cy, sy};
            const double gy2[3] = {1.0, flow ? cy : cy2, flow ? sy : sy2};
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    S.X[rho][i][3 * a + c] = gx[a] * gx2[c];
                    S.Y[rho][i][3 * a + c] = gy[a] * gy2[c];
                }
            if (flow) {
                // e(k + q/2) and e(k - q/2): cos(k +- q/2) = cos k cos q/2 -+ sin k sin q/2
                const double cxp = fma(cx, tq.cqx, -sx * tq.sqx), cxm = fma(cx, tq.cqx, sx * tq.sqx);
                S.CY[rho][i][0] = fma(cy, tq.cqy, -sy * tq.sqy);
                S.CY[rho][i][1] = fma(cy, tq.cqy, sy * tq.sqy);
                A1 = fma(tA, cxp, -lat.mu);
                B1 = fma(tB, cxp, tA);
                A2 = fma(tA, cxm, -lat.mu);
                B2 = fma(tB, cxm, tA);
            } else {
                S.CY[rho][i][0] = cy;
                S.CY[rho][i][1] = cy2;
                // x = e / 2T = A + B cos ky along row i, for k and for k' (for pp
                // the second energy enters with its sign flipped)
                const double h1 = B->inv2T, h2 = pp ? -B->inv2T : B->inv2T;
                A1 = fma(tA, cx, -lat.mu) * h1;
                B1 = fma(tB, cx, tA) * h1;
                A2 = fma(tA, cx2, -lat.mu) * h2;
                B2 = fma(tB, cx2, tA) * h2;
            }
        }
        __syncthreads();
        if (live) {
            double rf[9], rc[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) { rf[k] = 0.0; rc[k] = 0.0; }
#pragma unroll
            for (int j = 0; j < NF; ++j) {
                // OVERLAP: 1; bubbles: 2T F (1/2T is in the Jacobian); flow: dF/dOmega
                double F = 1.0;
                const double x1 = fma(B1, S.CY[rho][j][0], A1);
                const double x2 = fma(B2, S.CY[rho][j][1], A2);
                if (is_flow(kind))
                    F = flow_Fdot(x1, x2, B->T, kind == FLOW_PP);
                else if (kind != OVERLAP)
                    F = bubble_F2T(x1, x2, S.tab);
                const double wf = c_wf[v][j] * F;
#pragma unroll
                for (int k = 0; k < 9; ++k) rf[k] = fma(wf, S.Y[rho][j][k], rf[k]);
                if ((j & 1) == 0) {
                    const double wc = c_wc[v][j >> 1] * F;
#pragma unroll
                    for (int k = 0; k < 9; ++k) rc[k] = fma(wc, S.Y[rho][j][k], rc[k]);
                }
            }
            // the row's own rule weight (fine, and coarse on the even rows)
            // goes into its sums, so the moments below are plain dot products
            const double wr = c_wf[v][i];
#pragma unroll
            for (int k = 0; k < 9; ++k) S.Rf[rho][i][k] = wr * rf[k];
            if ((i & 1) == 0) {
                const double wrc = c_wc[v][i >> 1];
#pragma unroll
                for (int k = 0; k < 9; ++k) S.Rc[rho][i >> 1][k] = wrc * rc[k];
            }
        }
        __syncthreads();
        if (live) {
            // moments M[ac][bd]: the 81 (ac, bd) cells dealt over the region's
            // NF threads (all of them busy, rather than one thread per ac)
            for (int u = i; u < 81; u += NF) {
                const int ac = u / 9, bd = u - 9 * (u / 9);
                double mf = 0.0, mc = 0.0;
#pragma unroll
                for (int r = 0; r < NF; ++r) mf = fma(S.X[rho][r][ac], S.Rf[rho][r][bd], mf);
#pragma unroll
                for (int r = 0; r <= N; ++r) mc = fma(S.X[rho][2 * r][ac], S.Rc[rho][r][bd], mc);
                S.Mf[rho][ac][bd] = mf;
                S.Mc[rho][ac][bd] = mc;
            }
        }
        __syncthreads();
        if (live) {
            const double scale =
                ldexp(0.25, -2 * int(L)) * (kind == PH || kind == PP ? B->inv2T : 1.0);
            for (int p = i; p < P; p += NF) {
                const int l = B->lm[2 * p], m = B->lm[2 * p + 1];
                double q2 = 0.0, q1 = 0.0;
                if (l >= 0 && m >= 0 && l < w.nff && m < w.nff) {
                    for (int k1 = 0; k1 < c_ffn[l]; ++k1)
                        for (int k2 = 0; k2 < c_ffn[m]; ++k2) {
                            const double c = c_ffc[l][k1] * c_ffc[m][k2];
                            const int ac = 3 * c_ffa[l][k1] + c_ffa[m][k2];
                            const int bd = 3 * c_ffb[l][k1] + c_ffb[m][k2];
                            q2 = fma(c, S.Mf[rho][ac][bd], q2);
                            q1 = fma(c, S.Mc[rho][ac][bd], q1);
                        }
                }
                q2 *= scale;
                q1 *= scale;
                if (rule_q2) {
                    rule_q2[t * P + p] = q2;
                    rule_d[t * P + p] = q1 - q2;
                } else {
                    const size_t o = size_t(pos) * size_t(w.vstride) + size_t(p);
                    w.vval[cur][o] = q2;
                    w.verr[cur][o] = float(fabs(q1 - q2));
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// The FP32-pipe form of the shared-partition kernel (options.eval_fp32 with
// group_mode).  Same rule and data flow as k_eval_group, with every per-node,
// per-row and per-region quantity an unevaluated pair of FP32 numbers on the
// FP32 pipe (64x the FP64 pipe on this GPU): the node abscissae (rotations of
// the region centre), the reduced energies, the kernel F, the row sums, the
// moments, the pair combinations and the Jacobian.  FP64 remains for the two
// sincospi of the exact dyadic centre, the conversions of the per-region
// inputs, and each pair value's final conversion to FP64.
//
// The moments are taken in the Fourier basis phi = (1, cos k, sin k, cos 2k,
// sin 2k) of each direction instead of the nine products X_ac = g_a(k) g'_c(k')
// (g = (1, cos k, sin k) at k, g' the same at k' = k + q, or q - k for pp, or
// k for the flow kinds): every product is a fixed combination of the five
// (cos k cos k' = cos q (1 + cos 2k) / 2 - s sin q sin 2k / 2, ...), so a row
// needs 5 sums instead of 9 and a region 25 moments instead of 81, and the 81
// product moments follow from two small exact transforms per rule
// (ff_fourier_to_products).
template <int N>
struct GroupSmemF {
    static constexpr int NF = 2 * N + 1, R = GroupShape<N>::R;
    float2 X[R][NF][5];          // phi_u(kx_i) at the fine rows
    union {                      // the column data until every row is summed,
        struct {                 // then the row sums, then the x-transformed moments
            float2 Yf[R][NF][5];     // wf_j phi_v(ky_j)
            float2 Yc[R][N + 1][5];  // wc_j phi_v(ky_2j)
            float2 CY[R][NF][2];     // cos ky, cos ky' (flow kinds: cos(ky -+ qy/2))
        } c;
        struct {
            float2 Rf[R][NF][5];     // row sums with the row's fine weight
            float2 Rc[R][N + 1][5];  // coarse (even rows)
        } r;
        float2 T[R][2][9][5];        // G with the x index taken to X_ac (fine, coarse)
    } u;
    float2 G[R][2][5][5];        // Fourier moments (fine, coarse)
    float2 M[R][2][9][9];        // product moments M[ac][bd] (fine, coarse)
    float2 C[R][4];              // sin, cos of the region centre (x, y) times pi
    float2 Q[R][4];              // cos qx, sin qx, cos qy, sin qy (flow: of q/2)
    float2 H[R][2];              // 1/2T, T (Omega for the flow kinds)
    float2 tab[64];              // 2^(j/64)
    float2 wr[NF];               // fine weights
    float2 wrc[N + 1];           // coarse weights
    float2 lat[3];               // -2t, -4t', mu
};

__device__ __forceinline__ f2 ff_ld(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ float2 ff_st(f2 a) { return make_float2(a.hi, a.lo); }
// (c, s) rotated by the angle with cosine co and sine so
__device__ __forceinline__ void ff_rot(f2 c, f2 s, f2 co, f2 so, f2& c2, f2& s2)
{
    c2 = ff_sub(ff_mul(c, co), ff_mul(s, so));
    s2 = ff_add(ff_mul(s, co), ff_mul(c, so));
}

// Coefficients g_u of a function in the basis phi = (1, c, s, cos 2k, sin 2k)
// (c, s = cos k, sin k) to its products with (1, c, s) x (1, c', s'), index
// 3a + c, where (c', s') is (c, sg s) rotated by the angle with cosine cq and
// sine sq (sg = -1 for pp's k' = q - k).  With c^2 = (1 + cos 2k) / 2,
// s^2 = (1 - cos 2k) / 2 and s c = sin 2k / 2:
//   c'   = cq c - sg sq s           s'   = sq c + sg cq s
//   c c' = cq (1 + cos 2k)/2 - sg sq sin 2k/2
//   c s' = sq (1 + cos 2k)/2 + sg cq sin 2k/2
//   s c' = cq sin 2k/2 - sg sq (1 - cos 2k)/2
//   s s' = sq sin 2k/2 + sg cq (1 - cos 2k)/2
__device__ __forceinline__ void ff_fourier_to_products(const f2 g[5], f2 cq, f2 sq, bool flip,
                                                       f2 out[9])
{
    const f2 cs = flip ? ff_neg(cq) : cq, ss = flip ? ff_neg(sq) : sq;   // sg cq, sg sq
    const f2 hc = {0.5f * cq.hi, 0.5f * cq.lo}, hs = {0.5f * sq.hi, 0.5f * sq.lo};
    const f2 hcs = {0.5f * cs.hi, 0.5f * cs.lo}, hss = {0.5f * ss.hi, 0.5f * ss.lo};
    const f2 pl = ff_add(g[0], g[3]), mi = ff_sub(g[0], g[3]);
    out[0] = g[0];
    out[1] = ff_sub(ff_mul(cq, g[1]), ff_mul(ss, g[2]));
    out[2] = ff_add(ff_mul(sq, g[1]), ff_mul(cs, g[2]));
    out[3] = g[1];
    out[4] = ff_sub(ff_mul(hc, pl), ff_mul(hss, g[4]));
    out[5] = ff_add(ff_mul(hs, pl), ff_mul(hcs, g[4]));
    out[6] = g[2];
    out[7] = ff_sub(ff_mul(hc, g[4]), ff_mul(hss, mi));
    out[8] = ff_add(ff_mul(hs, g[4]), ff_mul(hcs, mi));
}

// KF: the kinds the launch may meet -- 0 any, 1 no flow kind, 2 flow kinds
// only -- so that a launch carries only the kernel F it needs (the row loop's
// code stays within the instruction cache).
template <int N, int KF>
__global__ void __launch_bounds__(GroupShape<N>::R * (2 * N + 1), 7)
k_eval_group_ff(Work w, Lattice lat, double* rule_q2, double* rule_d)
{
    constexpr int NF = 2 * N + 1, R = GroupShape<N>::R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GroupSmemF<N>& S = *reinterpret_cast<GroupSmemF<N>*>(smem_raw);
    const int v = rule_variant(N);
    const int cur = w.ls->cur;
    const int64_t n_eval = w.ls->n_eval;
    const int rho = threadIdx.x / NF, i = threadIdx.x % NF;
    if (threadIdx.x < 64) S.tab[threadIdx.x] = ff_st(ff_from(c_exp2d[threadIdx.x]));
    if (threadIdx.x < NF) S.wr[threadIdx.x] = ff_st(ff_from(c_wf[v][threadIdx.x]));
    if (threadIdx.x <= N) S.wrc[threadIdx.x] = ff_st(ff_from(c_wc[v][threadIdx.x]));
    if (threadIdx.x < 3)
        S.lat[threadIdx.x] = ff_st(ff_from(threadIdx.x == 0 ? -2.0 * lat.t
                                           : threadIdx.x == 1 ? -4.0 * lat.tp : lat.mu));
    for (int64_t chunk = blockIdx.x; chunk * R < n_eval; chunk += gridDim.x) {
        const int64_t t = chunk * R + rho;
        const bool live = t < n_eval;
        uint32_t pos = 0, g = 0, L = 0;
        int kind = PH, P = 0;
        const DevBatch* B = nullptr;
        f2 A1 = {0.0f, 0.0f}, B1 = A1, A2 = A1, B2 = A1;
        if (live) {
            const uint2 e = w.evl[t];
            pos = e.x;
            g = e.y;
            const uint64_t key = w.key[cur][pos];
            L = key_level(key);
            // the per-region inputs, one thread each: the exact dyadic centre
            // / pi = -1 + (2 ix + 1) 2^-L (x, then y), the transfer momentum,
            // the temperature
            if (i < 2) {
                const uint32_t ic = i == 0 ? key_ix(key) : key_iy(key);
                double sn, cs;
                sincospi(fma(double(2 * ic + 1), ldexp(1.0, -int(L)), -1.0), &sn, &cs);
                S.C[rho][2 * i] = ff_st(ff_from(sn));
                S.C[rho][2 * i + 1] = ff_st(ff_from(cs));
            } else if (i == 2) {
                const QTrig tq = w.trig[g];
                S.Q[rho][0] = ff_st(ff_from(tq.cqx));
                S.Q[rho][1] = ff_st(ff_from(tq.sqx));
                S.Q[rho][2] = ff_st(ff_from(tq.cqy));
                S.Q[rho][3] = ff_st(ff_from(tq.sqy));
            } else if (i == 3) {
                const DevBatch& Bt = w.batches[meta_batch(w.meta[g])];
                S.H[rho][0] = ff_st(ff_from(Bt.inv2T));
                S.H[rho][1] = ff_st(ff_from(Bt.T));
            }
        }
        __syncthreads();
        if (live) {
            const uint32_t mt = w.meta[g];
            B = &w.batches[meta_batch(mt)];
            kind = meta_kind(mt);
            P = B->npairs;
            const bool pp = kind == PP, flow = KF == 2 || (KF == 0 && is_flow(kind));
            const int ii = i <= N ? i : 2 * N - i;
            const f2 co = ff_from(c_co[v][L][ii]);
            const f2 so0 = ff_from(c_so[v][L][ii]);
            const f2 so = i <= N ? so0 : ff_neg(so0);
            const f2 cqx = ff_ld(S.Q[rho][0]), sqx = ff_ld(S.Q[rho][1]);
            const f2 cqy = ff_ld(S.Q[rho][2]), sqy = ff_ld(S.Q[rho][3]);
            // row i (x) and column i (y) of the fine grid
            f2 cx, sx, cy, sy;
            ff_rot(ff_ld(S.C[rho][1]), ff_ld(S.C[rho][0]), co, so, cx, sx);
            ff_rot(ff_ld(S.C[rho][3]), ff_ld(S.C[rho][2]), co, so, cy, sy);
            // the shifted k' (q + k: rotate by q; q - k: rotate -k by q);
            // flow kinds: both form factors at k
            f2 cx2 = cx, sx2 = sx, cy2 = cy, sy2 = sy;
            if (!flow) {
                if (pp) {
                    ff_rot(cx, ff_neg(sx), cqx, sqx, cx2, sx2);
                    ff_rot(cy, ff_neg(sy), cqy, sqy, cy2, sy2);
                } else {
                    ff_rot(cx, sx, cqx, sqx, cx2, sx2);
                    ff_rot(cy, sy, cqy, sqy, cy2, sy2);
                }
            }
            // the Fourier basis at row i (x) and column i (y)
            const f2 one = {1.0f, 0.0f};
            const f2 px[5] = {one, cx, sx, ff_mul(ff_sub(cx, sx), ff_add(cx, sx)),
                              ff_mul(f2{2.0f * sx.hi, 2.0f * sx.lo}, cx)};
            const f2 py[5] = {one, cy, sy, ff_mul(ff_sub(cy, sy), ff_add(cy, sy)),
                              ff_mul(f2{2.0f * sy.hi, 2.0f * sy.lo}, cy)};
            const f2 wf = ff_ld(S.wr[i]);
            const f2 wc = (i & 1) == 0 ? ff_ld(S.wrc[i >> 1]) : f2{0.0f, 0.0f};
#pragma unroll
            for (int u = 0; u < 5; ++u) {
                S.X[rho][i][u] = ff_st(px[u]);
                S.u.c.Yf[rho][i][u] = ff_st(ff_mul(wf, py[u]));
                if ((i & 1) == 0) S.u.c.Yc[rho][i >> 1][u] = ff_st(ff_mul(wc, py[u]));
            }
            const f2 tA = ff_ld(S.lat[0]), tB = ff_ld(S.lat[1]), nmu = ff_neg(ff_ld(S.lat[2]));
            if (flow) {
                // e(k + q/2) and e(k - q/2), tq the rotation by q/2
                f2 cxp, sxp, cxm, sxm, cyp, syp, cym, sym;
                ff_rot(cx, sx, cqx, sqx, cxp, sxp);
                ff_rot(cx, sx, cqx, ff_neg(sqx), cxm, sxm);
                ff_rot(cy, sy, cqy, sqy, cyp, syp);
                ff_rot(cy, sy, cqy, ff_neg(sqy), cym, sym);
                S.u.c.CY[rho][i][0] = ff_st(cyp);
                S.u.c.CY[rho][i][1] = ff_st(cym);
                A1 = ff_fma(tA, cxp, nmu);
                B1 = ff_fma(tB, cxp, tA);
                A2 = ff_fma(tA, cxm, nmu);
                B2 = ff_fma(tB, cxm, tA);
            } else {
                S.u.c.CY[rho][i][0] = ff_st(cy);
                S.u.c.CY[rho][i][1] = ff_st(cy2);
                // x = e / 2T = A + B cos ky along row i, for k and for k' (for pp
                // the second energy enters with its sign flipped)
                const f2 h1 = ff_ld(S.H[rho][0]), h2 = pp ? ff_neg(h1) : h1;
                A1 = ff_mul(ff_fma(tA, cx, nmu), h1);
                B1 = ff_mul(ff_fma(tB, cx, tA), h1);
                A2 = ff_mul(ff_fma(tA, cx2, nmu), h2);
                B2 = ff_mul(ff_fma(tB, cx2, tA), h2);
            }
        }
        __syncthreads();
        f2 rf[5], rc[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) { rf[k] = {0.0f, 0.0f}; rc[k] = {0.0f, 0.0f}; }
        if (live) {
            const f2 W = ff_ld(S.H[rho][1]);
            // one node (i, j): the kernel F once, then every row sum
            auto node = [&](int j, bool even) {
                const f2 x1 = ff_fma(B1, ff_ld(S.u.c.CY[rho][j][0]), A1);
                const f2 x2 = ff_fma(B2, ff_ld(S.u.c.CY[rho][j][1]), A2);
                f2 F = {1.0f, 0.0f};
                if (KF != 1 && is_flow(kind))
                    F = flow_Fdot_ff(x1, x2, W, kind == FLOW_PP);
                else if (KF != 2 && kind != OVERLAP)
                    F = bubble_F2T_ff(x1, x2, S.tab);
#pragma unroll
                for (int k = 0; k < 5; ++k) ff_acc(F, ff_ld(S.u.c.Yf[rho][j][k]), rf[k]);
                if (even) {
#pragma unroll
                    for (int k = 0; k < 5; ++k) ff_acc(F, ff_ld(S.u.c.Yc[rho][j >> 1][k]), rc[k]);
                }
            };
            // two columns per trip (even, then odd) keeps the coarse-rule
            // columns static without unrolling all 2N+1 nodes of the row: the
            // node is ~400 instructions, and a fully unrolled row overflows
            // the instruction cache; the last (even) column runs in the same
            // code under a uniform branch
#pragma unroll 1
            for (int j = 0; j < NF; j += 2) {
                node(j, true);
                if (j + 1 < NF) node(j + 1, false);
            }
        }
        // the row sums take the column data's memory: every row is done first
        __syncthreads();
        if (live) {
            // the row's own weight in float-float
            const f2 wr = ff_ld(S.wr[i]);
#pragma unroll
            for (int k = 0; k < 5; ++k)
                S.u.r.Rf[rho][i][k] = ff_st(ff_mul(wr, ff_fast(rf[k].hi, rf[k].lo)));
            if ((i & 1) == 0) {
                const f2 wrc = ff_ld(S.wrc[i >> 1]);
#pragma unroll
                for (int k = 0; k < 5; ++k)
                    S.u.r.Rc[rho][i >> 1][k] = ff_st(ff_mul(wrc, ff_fast(rc[k].hi, rc[k].lo)));
            }
        }
        __syncthreads();
        if (live) {
            // Fourier moments G[u][v]: the 25 cells dealt over the region's NF
            // threads, float-float dot products over the rows
            for (int c = i; c < 25; c += NF) {
                const int u = c / 5, v = c - 5 * (c / 5);
                f2 gf = {0.0f, 0.0f}, gc = {0.0f, 0.0f};
#pragma unroll 5
                for (int r = 0; r < NF; ++r)
                    ff_acc(ff_ld(S.X[rho][r][u]), ff_ld(S.u.r.Rf[rho][r][v]), gf);
#pragma unroll
                for (int r = 0; r <= N; ++r)
                    ff_acc(ff_ld(S.X[rho][2 * r][u]), ff_ld(S.u.r.Rc[rho][r][v]), gc);
                S.G[rho][0][u][v] = ff_st(ff_fast(gf.hi, gf.lo));
                S.G[rho][1][u][v] = ff_st(ff_fast(gc.hi, gc.lo));
            }
        }
        __syncthreads();
        // the rotation of k' and its orientation: (cos q, sin q) per direction
        // for ph / pp (pp: k' = q - k), none for the flow kinds (both form
        // factors at k)
        const bool flowk = live && (KF == 2 || (KF == 0 && is_flow(kind)));
        const bool flip = live && !flowk && kind == PP;
        const f2 one = {1.0f, 0.0f}, zero = {0.0f, 0.0f};
        if (live) {
            // x: each column v of G (per rule) to the nine X_ac
            for (int c = i; c < 10; c += NF) {
                const int rule = c / 5, v = c - 5 * (c / 5);
                f2 g[5], o[9];
#pragma unroll
                for (int u = 0; u < 5; ++u) g[u] = ff_ld(S.G[rho][rule][u][v]);
                ff_fourier_to_products(g, flowk ? one : ff_ld(S.Q[rho][0]),
                                       flowk ? zero : ff_ld(S.Q[rho][1]), flip, o);
#pragma unroll
                for (int ac = 0; ac < 9; ++ac) S.u.T[rho][rule][ac][v] = ff_st(o[ac]);
            }
        }
        __syncthreads();
        if (live) {
            // y: each row ac (per rule) to the nine Y_bd
            for (int c = i; c < 18; c += NF) {
                const int rule = c / 9, ac = c - 9 * (c / 9);
                f2 g[5], o[9];
#pragma unroll
                for (int v = 0; v < 5; ++v) g[v] = ff_ld(S.u.T[rho][rule][ac][v]);
                ff_fourier_to_products(g, flowk ? one : ff_ld(S.Q[rho][2]),
                                       flowk ? zero : ff_ld(S.Q[rho][3]), flip, o);
#pragma unroll
                for (int bd = 0; bd < 9; ++bd) S.M[rho][rule][ac][bd] = ff_st(o[bd]);
            }
        }
        __syncthreads();
        if (live) {
            // the Jacobian: 1/2T (ph, pp) in float-float times 4^-L / 4, an exact
            // power of two applied to both words
            const f2 jac = kind == PH || kind == PP ? ff_ld(S.H[rho][0]) : f2{1.0f, 0.0f};
            const float p2 = __int_as_float((125 - 2 * int(L)) << 23);
            for (int p = i; p < P; p += NF) {
                const int l = B->lm[2 * p], m = B->lm[2 * p + 1];
                f2 q2 = {0.0f, 0.0f}, q1 = {0.0f, 0.0f};
                if (l >= 0 && m >= 0 && l < w.nff && m < w.nff) {
                    for (int k1 = 0; k1 < c_ffn[l]; ++k1)
                        for (int k2 = 0; k2 < c_ffn[m]; ++k2) {
                            const f2 c = ff_ld(c_ffpair[l][k1][m][k2]);
                            const int ac = 3 * c_ffa[l][k1] + c_ffa[m][k2];
                            const int bd = 3 * c_ffb[l][k1] + c_ffb[m][k2];
                            ff_acc(c, ff_ld(S.M[rho][0][ac][bd]), q2);
                            ff_acc(c, ff_ld(S.M[rho][1][ac][bd]), q1);
                        }
                }
                q2 = ff_fast(q2.hi, q2.lo);
                q1 = ff_fast(q1.hi, q1.lo);
                // Q_2N and the embedded-rule difference Q_N - Q_2N; only the
                // value's conversion to FP64 leaves the FP32 pipe
                const f2 v = ff_mul(q2, jac), dq = ff_mul(ff_sub(q1, q2), jac);
                const double v2 = double(__fmul_rn(v.hi, p2)) + double(__fmul_rn(v.lo, p2));
                if (rule_q2) {
                    rule_q2[t * P + p] = v2;
                    rule_d[t * P + p] =
                        double(__fmul_rn(dq.hi, p2)) + double(__fmul_rn(dq.lo, p2));
                } else {
                    const size_t o = size_t(pos) * size_t(w.vstride) + size_t(p);
                    w.vval[cur][o] = v2;
                    w.verr[cur][o] = fabsf(__fmul_rn(dq.hi, p2));
                }
            }
        }
        __syncthreads();
    }
}

template <int N>
static cudaError_t group_attr()
{
    cudaError_t e = cudaFuncSetAttribute(k_eval_group<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(sizeof(GroupSmem<N>)));
    for (int kf = 0; kf < 3 && e == cudaSuccess; ++kf)
        e = cudaFuncSetAttribute(kf == 0 ? k_eval_group_ff<N, 0>
                                 : kf == 1 ? k_eval_group_ff<N, 1> : k_eval_group_ff<N, 2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(sizeof(GroupSmemF<N>)));
    return e;
}

static cudaError_t group_kernel_attributes()
{
    cudaError_t e = group_attr<4>();
    if (e == cudaSuccess) e = group_attr<6>();
    if (e == cudaSuccess) e = group_attr<8>();
    if (e == cudaSuccess) e = group_attr<10>();
    if (e == cudaSuccess) e = group_attr<12>();
    return e;
}

template <int N>
static void group_launch(const Work& w, int64_t hint_eval, int64_t cap, int fp32, Lattice lat,
                         cudaStream_t s, double* rule_q2, double* rule_d)
{
    constexpr int R = GroupShape<N>::R;
    const int64_t blocks = std::min<int64_t>((hint_eval + R - 1) / R, cap);
    const dim3 grid(static_cast<unsigned>(blocks)), block(R * (2 * N + 1));
    const size_t sm = sizeof(GroupSmemF<N>);
    if (fp32 && w.kinds == 1)
        k_eval_group_ff<N, 1><<<grid, block, sm, s>>>(w, lat, rule_q2, rule_d);
    else if (fp32 && w.kinds == 2)
        k_eval_group_ff<N, 2><<<grid, block, sm, s>>>(w, lat, rule_q2, rule_d);
    else if (fp32)
        k_eval_group_ff<N, 0><<<grid, block, sm, s>>>(w, lat, rule_q2, rule_d);
    else
        k_eval_group<N><<<int(blocks), R * (2 * N + 1), sizeof(GroupSmem<N>), s>>>(
            w, lat, rule_q2, rule_d);
}

cudaError_t launch_eval_group(const Work& w, int64_t hint_eval, int rule_n, int fp32, Lattice lat,
                              cudaStream_t s, double* rule_q2, double* rule_d, int max_blocks)
{
    if (hint_eval <= 0) return cudaSuccess;
    const int64_t cap = max_blocks > 0 ? max_blocks : 152 * 32;
    switch (rule_n) {
    case 4: group_launch<4>(w, hint_eval, cap, fp32, lat, s, rule_q2, rule_d); break;
    case 6: group_launch<6>(w, hint_eval, cap, fp32, lat, s, rule_q2, rule_d); break;
    case 8: group_launch<8>(w, hint_eval, cap, fp32, lat, s, rule_q2, rule_d); break;
    case 10: group_launch<10>(w, hint_eval, cap, fp32, lat, s, rule_q2, rule_d); break;
    default: group_launch<12>(w, hint_eval, cap, fp32, lat, s, rule_q2, rule_d); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_eval(const Work& w, int64_t hint_eval, int rule_n, int fp32, Lattice lat,
                        cudaStream_t s, cudaEvent_t mid)
{
    if (hint_eval <= 0) return cudaSuccess;
    const int threads = 128;
    int64_t blocks = (hint_eval + threads - 1) / threads;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (fp32) {
        const int dblocks = int(std::min<int64_t>((hint_eval + kYsStride - 1) / kYsStride, 152 * 48));
        if (rule_n == 4) k_eval_fp32<4><<<int(blocks), threads, 0, s>>>(w, lat);
        else             k_eval_fp32<6><<<int(blocks), threads, 0, s>>>(w, lat);
        if (mid) {
            const cudaError_t e = cudaEventRecord(mid, s);
            if (e != cudaSuccess) return e;
        }
        if (rule_n == 4) k_eval_df<4><<<dblocks, kYsStride, 0, s>>>(w, lat);
        else             k_eval_df<6><<<dblocks, kYsStride, 0, s>>>(w, lat);
    } else {
        if (rule_n == 4) k_eval_fp64<4><<<int(blocks), threads, 0, s>>>(w, lat);
        else             k_eval_fp64<6><<<int(blocks), threads, 0, s>>>(w, lat);
    }
    return cudaGetLastError();
}

}  // namespace paid
