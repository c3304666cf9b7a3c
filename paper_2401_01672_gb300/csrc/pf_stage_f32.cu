// Stage kernels and launchers, field type float (the binary32-field form; the state stays binary64).
// The binary64 form is compiled in pf_stage_f64.cu from the same templates.
#include "pf_stage.cuh"

namespace pfgb {

cudaError_t launch_stage_f32(int model, int rx, int stage, const StageArgs<float>& a, int by, cudaStream_t s) {
    return launch_stage_t<float>(model, rx, stage, a, by, s);
}

cudaError_t launch_batch_stage_f32(int model, int rx, int stage, const StageArgs<float>* args, const BatchPlan* plan,
                                   const int4* tg, int by, int blocks, cudaStream_t s) {
    return launch_batch_stage_t<float>(model, rx, stage, args, plan, tg, by, blocks, s);
}

}  // namespace pfgb
