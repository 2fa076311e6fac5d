// Thermochemistry kernels of one precision family, RT_FP64 with smoothed RT (Sec. 3.4): the
// instantiations of thermo_kernels.cuh for every group count, one family
// per translation unit so that they compile in parallel.
#include "thermo_kernels.cuh"

namespace rtgb {

cudaError_t thermo_dispatch_f64_sm(const ThermoParams &tp, int G, const double *nH, double *xHII, double *xHeII, double *xHeIII,
               double *T, double *N, double *F, double *Npre, double *Fpre, int32_t *subcycles, Queue q, unsigned *status,
               int n_sm, cudaStream_t s, cudaEvent_t *ev)
{
    return dispatch_g<double, false, true>(tp, G, nH, xHII, xHeII, xHeIII, T, N, F, Npre, Fpre, subcycles, q, status, n_sm, s,
                                  ev);
}

}  // namespace rtgb
