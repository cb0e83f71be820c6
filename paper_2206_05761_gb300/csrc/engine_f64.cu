// 64-bit instantiation of the HWFV1 engine (the parity path).
#include "engine.cuh"

namespace hwfv1 {
Engine* make_engine_f64(const hwfv1_problem& spec, cudaStream_t stream) {
    return new EngineT<double>(spec, stream);
}
}  // namespace hwfv1
