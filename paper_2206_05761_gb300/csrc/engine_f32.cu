// 32-bit instantiation of the HWFV1 engine.
#include "engine.cuh"

namespace hwfv1 {
Engine* make_engine_f32(const hwfv1_problem& spec, cudaStream_t stream) {
    return new EngineT<float>(spec, stream);
}
}  // namespace hwfv1
