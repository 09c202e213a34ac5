// kernels.h -- host launchers of the CUDA kernels in kernels.cu.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "tn_internal.h"

namespace tn {

enum Dtype { DT_I32 = 1, DT_F32 = 2 };

// A batch of B instances sharing one plan: instance b uses the arena slice
// at b * ib bytes and the couplings J + b * jstride, h + b * hstride.
struct Batch {
  int B = 1;
  int64_t ib = 0, jstride = 0, hstride = 0;
};

// Streaming multiprocessors of the current device (queried once per device).
int num_sms();

// Leaves (Sec. II bond / vertex tensors).  x: base of the value arena (bytes),
// counts: when P > 0 every leaf element gets count 1 in each residue plane
// (planes of rbytes = 8- or 4-byte residues).
cudaError_t launch_leaves(Dtype dt, int q, const LeafDesc *d_leaves, int nleaves, const float *J,
                          const float *h, char *arena, int P, int rbytes, const Batch &bt,
                          cudaStream_t st);

// Gate contraction (small B); xA/xB/xC value pointers, nA/nB/nC plane-0
// pointers (counting only).
cudaError_t launch_gate(Dtype dt, const GateParams &p, const void *xA, const void *xB, void *xC,
                        const uint64_t *nA, const uint64_t *nB, uint64_t *nC, const PrimeSet &ps,
                        const Batch &bt, cudaStream_t st);

// Counting gate contraction with compile-time (K, N, planes) forms for 4-byte
// residue planes (gate_count_*.cu); false when the step has no such form (the
// generic kernel runs it).
bool launch_gate_tc_i32(const GateParams &p, const void *A, const void *B, void *C,
                        const uint32_t *nA, const uint32_t *nB, uint32_t *nC, const PrimeSet &ps,
                        const Batch &bt, cudaStream_t st);
bool launch_gate_tc_f32(const GateParams &p, const void *A, const void *B, void *C,
                        const uint32_t *nA, const uint32_t *nB, uint32_t *nC, const PrimeSet &ps,
                        const Batch &bt, cudaStream_t st);

// Register-tiled max-plus GEMM (128 x 128 tiles, cp.async staging), values only.
// The tile configuration of a shape class is chosen by timing the candidates
// on its first launch outside stream capture (set_gemm_autotune(false) on the
// calling thread skips that and uses the default).
cudaError_t launch_mpgemm(Dtype dt, const GemmParams &p, const void *A, const void *B, void *C,
                          const Batch &bt, cudaStream_t st);
// returns the previous setting of the calling thread
bool set_gemm_autotune(bool on);
// Residue planes of a counting GEMM whose values C were produced already.
cudaError_t launch_gemm_count(Dtype dt, const GemmParams &p, const void *xA, const void *xB,
                              const void *xC, const uint64_t *nA, const uint64_t *nB, uint64_t *nC,
                              const PrimeSet &ps, const Batch &bt, cudaStream_t st);

// Permutation of a tensor (values and, when P > 0, its residue planes).
cudaError_t launch_permute(const PermParams &p, const void *xin, void *xout, const uint64_t *nin,
                           uint64_t *nout, const Batch &bt, cudaStream_t st);

// Argmax traceback over steps [0, nsteps) of d_steps (Sec. III).
// *err is set to 1 if a step meets an unassigned spin (a planning error).
// Records with chain >= 0 refer to d_chains; smem: dynamic shared memory for
// the largest chain record (trace_smem_bytes).
// The spin state (nspins int8) is staged in shared memory during the walk.
cudaError_t launch_trace(Dtype dt, int q, const TraceStep *d_steps, int nsteps,
                         const ChainTrace *d_chains, size_t smem, const char *arena, int8_t *state,
                         int nspins, int *err, const Batch &bt, cudaStream_t st);
size_t trace_smem_bytes(const ChainParams &p, size_t elem);

// Fused gate chain over tiles of the big tensor (values; planes when P > 0).
cudaError_t launch_chain(Dtype dt, const ChainParams &p, const char *arena, const void *Ax,
                         const uint64_t *An, void *Cx, uint64_t *Cn, const PrimeSet &ps,
                         const Batch &bt, cudaStream_t st);
size_t chain_smem_bytes(const ChainParams &p, size_t elem);

// dE/dJ and dE/dh at the traced state.
cudaError_t launch_grad(int q, int n, int m, const int32_t *eu, const int32_t *ev,
                        const int8_t *state, float *dJ, float *dh, int B, cudaStream_t st);

// Convert a state (indices) to the +-1 / 0..q-1 convention of tn_config.
cudaError_t launch_state_out(int q, int n, const int8_t *state, int8_t *out, int B,
                             cudaStream_t st);

// Static scratch of tn_energy_noalloc (noalloc.cu): its size, its device
// address on the current device (looked up once per device), and the kernel
// writing E = -root as float.
size_t noalloc_scratch_bytes();
cudaError_t noalloc_scratch(char **ptr);
cudaError_t launch_energy_out(Dtype dt, const void *root, float *E, cudaStream_t st);
// Leaves of tn_energy_noalloc from host descriptors passed as kernel
// parameters (no device copy of the descriptors; values only).
cudaError_t launch_leaves_param(Dtype dt, int q, const LeafDesc *leaves, int nleaves,
                                const float *J, const float *h, char *scratch, cudaStream_t st);

}  // namespace tn
