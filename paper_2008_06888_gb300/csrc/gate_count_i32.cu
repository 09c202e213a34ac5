// gate_count_i32.cu -- the int32_t instantiations of the counting gate forms
// (gate_count.cuh).
#include "gate_count.cuh"

namespace tn {

bool launch_gate_tc_i32(const GateParams &p, const void *A, const void *B, void *C,
                         const uint32_t *nA, const uint32_t *nB, uint32_t *nC, const PrimeSet &ps,
                         const Batch &bt, cudaStream_t st) {
  return launch_gate_tc_typed<int32_t>(p, (const int32_t *)A, (const int32_t *)B, (int32_t *)C, nA, nB, nC, ps, bt,
                                  st);
}

}  // namespace tn
