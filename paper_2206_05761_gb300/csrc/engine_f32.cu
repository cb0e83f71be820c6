// 32-bit instantiation of the HWFV1 engine.
#include "batch.cuh"

namespace hwfv1 {
Engine* make_engine_f32(const hwfv1_problem& spec, cudaStream_t stream) {
    return new EngineT<float>(spec, stream);
}
Batch* make_batch_f32(const hwfv1_problem* specs, int n, cudaStream_t stream) {
    return new BatchT<float>(specs, n, stream);
}
}  // namespace hwfv1
