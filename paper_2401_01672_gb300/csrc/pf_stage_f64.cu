// Stage kernels and launchers, field type double (the binary64 form).  The binary32 form is compiled in
// pf_stage_f32.cu from the same templates, so that the two translation units build in parallel.
#include "pf_stage.cuh"

namespace pfgb {

cudaError_t launch_stage_f64(int model, int rx, int stage, const StageArgs<double>& a, int by, cudaStream_t s) {
    return launch_stage_t<double>(model, rx, stage, a, by, s);
}

cudaError_t launch_batch_stage_f64(int model, int rx, int stage, const StageArgs<double>* args, const BatchPlan* plan,
                                   const int4* tg, int by, int blocks, cudaStream_t s) {
    return launch_batch_stage_t<double>(model, rx, stage, args, plan, tg, by, blocks, s);
}

}  // namespace pfgb
