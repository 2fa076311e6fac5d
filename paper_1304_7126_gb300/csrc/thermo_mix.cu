// RT_MIXED thermochemistry launcher: FP32 photon state, FP64
// thermochemistry (kernels in thermo_kernels.cuh).
#include "thermo_kernels.cuh"

namespace rtgb {

cudaError_t launch_thermo_mixed(const ThermoParams &tp, int G, bool rates32, const double *nH, double *xHII,
                                double *xHeII, double *xHeIII, double *T, float *N, float *F, float *Npre,
                                float *Fpre, int32_t *subcycles, Queue q, unsigned *status, int n_sm, cudaStream_t s,
                                cudaEvent_t *ev)
{
    if (rates32) return launch_thermo_mixed32(tp, G, nH, xHII, xHeII, xHeIII, T, N, F, Npre, Fpre, subcycles, q,
                                              status, n_sm, s, ev);
    if (Npre)
        return dispatch_g<float, false, true>(tp, G, nH, xHII, xHeII, xHeIII, T, N, F, Npre, Fpre, subcycles, q,
                                              status, n_sm, s, ev);
    return dispatch_g<float, false, false>(tp, G, nH, xHII, xHeII, xHeIII, T, N, F, nullptr, nullptr, subcycles, q,
                                           status, n_sm, s, ev);
}

}  // namespace rtgb
