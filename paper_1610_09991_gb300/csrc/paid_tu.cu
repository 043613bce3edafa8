// Truncated-unity products of the flow equations (Eqs. matmul-P, matmul-C,
// matmul-D of Sec. 2): for every transfer momentum l, with X the scale
// derivatives of the pp and ph form-factor bubbles (nff x nff, the output
// order of a batch with all nff^2 pairs) and V^P, V^C, V^D the couplings,
//   dP = V^P X^pp V^P,   dC = -V^C X^ph V^C,
//   dD = 2 V^D X^ph V^D - V^C X^ph V^D - V^D X^ph V^C.
// One block per l: the five matrices in shared memory, the three left
// products V X once, then the right products; FP64 throughout.
#include "paid_internal.cuh"

namespace paid {

constexpr int kTuMax = 9;

__global__ void __launch_bounds__(128)
k_tu_rhs(int nq, int n, const double* VP, const double* VC, const double* VD, const double* Xpp,
         const double* Xph, double* dP, double* dC, double* dD)
{
    __shared__ double vp[kTuMax][kTuMax], vc[kTuMax][kTuMax], vd[kTuMax][kTuMax];
    __shared__ double xpp[kTuMax][kTuMax], xph[kTuMax][kTuMax];
    __shared__ double tp[kTuMax][kTuMax], tc[kTuMax][kTuMax], td[kTuMax][kTuMax];
    const int nn = n * n;
    for (int l = blockIdx.x; l < nq; l += gridDim.x) {
        const size_t o = size_t(l) * nn;
        for (int t = threadIdx.x; t < nn; t += blockDim.x) {
            const int a = t / n, b = t % n;
            vp[a][b] = VP[o + t];
            vc[a][b] = VC[o + t];
            vd[a][b] = VD[o + t];
            xpp[a][b] = Xpp[o + t];
            xph[a][b] = Xph[o + t];
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nn; t += blockDim.x) {
            const int a = t / n, b = t % n;
            double sp = 0.0, sc = 0.0, sd = 0.0;
            for (int i = 0; i < n; ++i) {
                sp = fma(vp[a][i], xpp[i][b], sp);
                sc = fma(vc[a][i], xph[i][b], sc);
                sd = fma(vd[a][i], xph[i][b], sd);
            }
            tp[a][b] = sp;   // V^P X^pp
            tc[a][b] = sc;   // V^C X^ph
            td[a][b] = sd;   // V^D X^ph
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nn; t += blockDim.x) {
            const int a = t / n, b = t % n;
            double p = 0.0, c = 0.0, d = 0.0;
            for (int j = 0; j < n; ++j) {
                p = fma(tp[a][j], vp[j][b], p);
                c = fma(tc[a][j], vc[j][b], c);
                d = fma(2.0 * td[a][j], vd[j][b], d);
                d = fma(-tc[a][j], vd[j][b], d);
                d = fma(-td[a][j], vc[j][b], d);
            }
            dP[o + t] = p;
            dC[o + t] = -c;
            dD[o + t] = d;
        }
        __syncthreads();
    }
}

cudaError_t launch_tu_rhs(int nq, int n, const double* VP, const double* VC, const double* VD,
                          const double* Xpp, const double* Xph, double* dP, double* dC,
                          double* dD, cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    const int blocks = nq < 152 * 16 ? nq : 152 * 16;
    k_tu_rhs<<<blocks, 128, 0, s>>>(nq, n, VP, VC, VD, Xpp, Xph, dP, dC, dD);
    return cudaGetLastError();
}

}  // namespace paid
