// Host build of the CUDA library's constitutive arithmetic (the functions
// the kernels call, compiled for the CPU) so that a CPU test can compare it
// with the FP64 oracle. Test infrastructure only.
#include "../../paper_2510_17335_gb300/csrc/mpm_device.cuh"

using namespace mpm;

template <typename T>
static void adjoint(const double* Ft_in, double mu, double lam, double alpha, double smin, const double* gFn_in,
                    const double* gtau_in, double* Fn_out, double* tau_out, double* gFt_out, double* gpar, int* kase) {
    T Ft[3][3], gFn[3][3], gtau[3][3], Fn[3][3], tau[3][3], gFt[3][3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            Ft[a][b] = (T)Ft_in[3 * a + b];
            gFn[a][b] = (T)gFn_in[3 * a + b];
            gtau[a][b] = (T)gtau_in[3 * a + b];
        }
    const T beta = (T)((3.0 * lam + 2.0 * mu) / (2.0 * mu) * alpha);
    Spectral<T> S;
    constitutive_spectral<T>(Ft, (T)mu, (T)lam, beta, (T)smin, S);
    spectral_outputs<T, T>(S, Fn, tau);
    T gm = 0, gl = 0, ga = 0;
    constitutive_adjoint_spectral<T>(S, (T)mu, (T)lam, (T)alpha, beta, (T)smin, gFn, gtau, gFt, gm, gl, ga);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            Fn_out[3 * a + b] = Fn[a][b];
            tau_out[3 * a + b] = tau[a][b];
            gFt_out[3 * a + b] = gFt[a][b];
        }
    gpar[0] = gm;
    gpar[1] = gl;
    gpar[2] = ga;
    *kase = S.kase;
}

extern "C" void hm_constitutive_adjoint(int fp64, const double* Ft, double mu, double lam, double alpha, double smin,
                                        const double* gFn, const double* gtau, double* Fn, double* tau, double* gFt,
                                        double* gpar, int* kase) {
    if (fp64)
        adjoint<double>(Ft, mu, lam, alpha, smin, gFn, gtau, Fn, tau, gFt, gpar, kase);
    else
        adjoint<float>(Ft, mu, lam, alpha, smin, gFn, gtau, Fn, tau, gFt, gpar, kase);
}
