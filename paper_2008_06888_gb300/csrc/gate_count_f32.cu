// gate_count_f32.cu -- the float instantiations of the counting gate forms
// (gate_count.cuh).
#include "gate_count.cuh"

namespace tn {

bool launch_gate_tc_f32(const GateParams &p, const void *A, const void *B, void *C,
                         const uint32_t *nA, const uint32_t *nB, uint32_t *nC, const PrimeSet &ps,
                         const Batch &bt, cudaStream_t st) {
  return launch_gate_tc_typed<float>(p, (const float *)A, (const float *)B, (float *)C, nA, nB, nC, ps, bt,
                                  st);
}

}  // namespace tn
