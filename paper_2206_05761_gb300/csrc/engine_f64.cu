// 64-bit instantiation of the HWFV1 engine (the parity path).
#include "batch.cuh"

namespace hwfv1 {
Engine* make_engine_f64(const hwfv1_problem& spec, cudaStream_t stream) {
    return new EngineT<double>(spec, stream);
}
Batch* make_batch_f64(const hwfv1_problem* specs, int n, cudaStream_t stream) {
    return new BatchT<double>(specs, n, stream);
}
}  // namespace hwfv1
