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
#include <cmath>
#include <cstdio>

#include "paid_internal.cuh"

namespace paid {

// rule variant 0: N = 4 (5 x 5 coarse inside 9 x 9 fine); 1: N = 6 (7 inside 13)
__constant__ double c_wf[2][2 * kMaxRuleN + 1];   // fine CC weights on [-1, 1]
__constant__ double c_wc[2][kMaxRuleN + 1];       // coarse CC weights
__constant__ double c_t[2][2 * kMaxRuleN + 1];    // fine nodes t_i = cos(i pi / 2N)
__constant__ double c_co[2][kMaxLevel + 1][kMaxRuleN + 1];  // cos(pi 2^-L t_i), i <= N
__constant__ double c_so[2][kMaxLevel + 1][kMaxRuleN + 1];  // sin(pi 2^-L t_i)
__constant__ double c_ff[9][3][3];                // f_n = sum_ab C[a][b] X_a Y_b

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

cudaError_t init_rule_tables(int device)
{
    static bool done[64] = {false};
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (done[device]) return cudaSuccess;
    double wf[2][2 * kMaxRuleN + 1] = {}, wc[2][kMaxRuleN + 1] = {}, t[2][2 * kMaxRuleN + 1] = {};
    double co[2][kMaxLevel + 1][kMaxRuleN + 1] = {}, so[2][kMaxLevel + 1][kMaxRuleN + 1] = {};
    const int Ns[2] = {4, 6};
    for (int v = 0; v < 2; ++v) {
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
    cudaError_t e;
    if ((e = cudaMemcpyToSymbol(c_wf, wf, sizeof(wf))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_wc, wc, sizeof(wc))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_t, t, sizeof(t))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_co, co, sizeof(co))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_so, so, sizeof(so))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_ff, ff, sizeof(ff))) != cudaSuccess) return e;
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

template <int N>
__global__ void __launch_bounds__(128) k_eval_fp64(Work w, int cur, int64_t n_eval, Lattice lat)
{
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
    }
}

cudaError_t launch_eval(const Work& w, int cur, int64_t n_eval, int rule_n, int fp32,
                        Lattice lat, cudaStream_t s)
{
    (void)fp32;
    if (n_eval <= 0) return cudaSuccess;
    const int threads = 128;
    int64_t blocks = (n_eval + threads - 1) / threads;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (rule_n == 4)
        k_eval_fp64<4><<<int(blocks), threads, 0, s>>>(w, cur, n_eval, lat);
    else
        k_eval_fp64<6><<<int(blocks), threads, 0, s>>>(w, cur, n_eval, lat);
    return cudaGetLastError();
}

}  // namespace paid
