// Thermochemistry kernels of one precision family, RT_MIXED (FP32 photon state, FP64 thermochemistry): the
// instantiations of thermo_kernels.cuh for every group count, one family
// per translation unit so that they compile in parallel.
#include "thermo_kernels.cuh"

namespace rtgb {

cudaError_t thermo_dispatch_mix(const ThermoParams &tp, int G, const double *nH, double *xHII, double *xHeII, double *xHeIII,
               double *T, float *N, float *F, float *Npre, float *Fpre, int32_t *subcycles, Queue q, unsigned *status,
               int n_sm, cudaStream_t s, cudaEvent_t *ev)
{
    return dispatch_g<float, false, false>(tp, G, nH, xHII, xHeII, xHeIII, T, N, F, Npre, Fpre, subcycles, q, status, n_sm, s,
                                  ev);
}

}  // namespace rtgb
