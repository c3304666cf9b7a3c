// Instantiations and launcher of the stage kernels, field type double.
#include "pf_stage.cuh"

namespace pfgb {

namespace {
using T = double;

template <int MODEL, int RX, int BY>
cudaError_t launch_by(int stage, const StageArgs<T>& a, cudaStream_t s) {
    const int n1 = a.cf.n1, n2 = a.cf.n2, n3 = a.cf.n3;
    dim3 block(TX, BY);
    dim3 grid((n1 + TX - 1) / TX, (n2 + BY - 1) / BY, (n3 + a.zc - 1) / a.zc);
    switch (stage) {
        case 0: stage_kernel<MODEL, RX, T, T, 0, BY><<<grid, block, 0, s>>>(a); break;
        case 1: stage_kernel<MODEL, RX, T, double, 1, BY><<<grid, block, 0, s>>>(a); break;
        case 2: stage_kernel<MODEL, RX, T, T, 2, BY><<<grid, block, 0, s>>>(a); break;
        case 3: stage_kernel<MODEL, RX, T, T, 3, BY><<<grid, block, 0, s>>>(a); break;
        case 4: stage_kernel<MODEL, RX, T, T, 4, BY><<<grid, block, 0, s>>>(a); break;
        case 5: stage_kernel<MODEL, RX, T, T, 5, BY><<<grid, block, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

template <int MODEL, int RX>
cudaError_t launch_m(int stage, const StageArgs<T>& a, int by, cudaStream_t s) {
    switch (by) {
        case 4: return launch_by<MODEL, RX, 4>(stage, a, s);
        case 8: return launch_by<MODEL, RX, 8>(stage, a, s);
        case 16: return launch_by<MODEL, RX, 16>(stage, a, s);
        default: return cudaErrorInvalidValue;
    }
}
template <int MODEL, int RX, int BY>
cudaError_t batch_by(int stage, const StageArgs<T>* args, const BatchPlan* plan, const int4* tg, int blocks,
                     cudaStream_t s) {
    dim3 block(TX, BY);
    switch (stage) {
        case 1: batch_stage_kernel<MODEL, RX, T, double, 1, BY><<<blocks, block, 0, s>>>(args, plan, tg); break;
        case 2: batch_stage_kernel<MODEL, RX, T, T, 2, BY><<<blocks, block, 0, s>>>(args, plan, tg); break;
        case 3: batch_stage_kernel<MODEL, RX, T, T, 3, BY><<<blocks, block, 0, s>>>(args, plan, tg); break;
        case 4: batch_stage_kernel<MODEL, RX, T, T, 4, BY><<<blocks, block, 0, s>>>(args, plan, tg); break;
        case 5: batch_stage_kernel<MODEL, RX, T, T, 5, BY><<<blocks, block, 0, s>>>(args, plan, tg); break;
        default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

template <int MODEL, int RX>
cudaError_t batch_m(int stage, const StageArgs<T>* args, const BatchPlan* plan, const int4* tg, int by, int blocks,
                    cudaStream_t s) {
    switch (by) {
        case 4: return batch_by<MODEL, RX, 4>(stage, args, plan, tg, blocks, s);
        case 8: return batch_by<MODEL, RX, 8>(stage, args, plan, tg, blocks, s);
        case 16: return batch_by<MODEL, RX, 16>(stage, args, plan, tg, blocks, s);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

cudaError_t launch_batch_stage_f64(int model, int rx, int stage, const StageArgs<T>* args, const BatchPlan* plan,
                                   const int4* tg, int by, int blocks, cudaStream_t s) {
    if (model == M_FULL) return rx == R_GRADP ? batch_m<M_FULL, R_GRADP>(stage, args, plan, tg, by, blocks, s)
                                              : batch_m<M_FULL, R_SIGMA>(stage, args, plan, tg, by, blocks, s);
    if (model == M_TEMP) return batch_m<M_TEMP, R_SIGMA>(stage, args, plan, tg, by, blocks, s);
    if (model == M_MICRO) return rx == R_GRADP ? batch_m<M_MICRO, R_GRADP>(stage, args, plan, tg, by, blocks, s)
                                               : batch_m<M_MICRO, R_SIGMA>(stage, args, plan, tg, by, blocks, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_stage_f64(int model, int rx, int stage, const StageArgs<T>& a, int by, cudaStream_t s) {
    if (a.zc <= 0) return cudaErrorInvalidValue;
    if (model == M_FULL) return rx == R_GRADP ? launch_m<M_FULL, R_GRADP>(stage, a, by, s)
                                              : launch_m<M_FULL, R_SIGMA>(stage, a, by, s);
    if (model == M_TEMP) return launch_m<M_TEMP, R_SIGMA>(stage, a, by, s);
    if (model == M_MICRO) return rx == R_GRADP ? launch_m<M_MICRO, R_GRADP>(stage, a, by, s)
                                               : launch_m<M_MICRO, R_SIGMA>(stage, a, by, s);
    return cudaErrorInvalidValue;
}

}  // namespace pfgb
