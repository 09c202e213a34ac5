// jit.h -- register chains compiled at run time.
//
// A register chain (q = 2, values, folded table gates) is a fixed sequence of
// table gates over the 2^RB register elements of a thread.  For large chains
// the program builder asks for a kernel specialised to that sequence: the
// gates, the register-leg offsets and the outer-index decoding become
// constants, so the chain runs as straight-line code without per-gate
// dispatch.  Kernels are compiled with NVRTC for sm_103a (one program per
// chain, in parallel), loaded with cudaLibraryLoadData and cached in memory
// and on disk by a hash of their source.
#pragma once
#include <string>
#include <vector>

#include "kernels.h"
#include "tn_internal.h"

namespace tn {

// Kernel handles (cudaKernel_t as const void *) for every chain that is
// worth compiling; nullptr elsewhere (the interpreting kernel runs those).
// Returns false with *err set if compilation or loading failed.
bool jit_chains(const std::vector<ChainParams> &chains, Dtype dt, std::vector<const void *> *out,
                std::string *err);

// Coalesced tile copies of a compiled chain with RB register legs (5 or 6),
// for one layout (input: hi = hi_in, output: hi = hi_out; a register leg with
// offset 0 there is not a leg of that layout).  A warp's tile is its 32 outer
// indices x 2^nreg register states; tile word bit j sits at memory position
// tpos[j] (tpos[j] == j for j < 5).  Word lane + 32 i lies at the warp's tile
// base + lane + off_i and in shared-memory slot D_lane ^ D_i (tile_word:
// D_i, off_i; D_lane = XOR_j<5 {cbit[j] : bit j of lane}); the thread of lane
// finds register state e at slot tile_slot(lane, e).
// Slots: the a (<= 2) register legs at memory positions 0..a-1 ("low" legs)
// are slot bits 0..a-1, the lane (XOR a swizzle of the other register bits)
// slot bits a..a+4 and the other register bits the bits above, so that a
// thread moves the 2^a states that differ in its low legs with one vector
// access and the tile copies stay vector copies too.
struct TileMap {
  int nreg = 0;                       // register legs of this layout
  int a = 0;                          // low register legs
  int rbit[6] = {0, 0, 0, 0, 0, 0};   // their bits in the register state index
  int gbit[6] = {0, 0, 0, 0, 0, 0};   // lane swizzle of each of them
  int lowbit[6] = {-1, -1, -1, -1, -1, -1};   // slot bit of a low leg
  int hibit[6] = {-1, -1, -1, -1, -1, -1};    // bit above the lane of another leg
  std::vector<int> cbit;
  std::vector<int> tpos;
};
bool tile_map(const ChainParams &p, const int64_t *hi, TileMap *tm);
int tile_slot(const TileMap &tm, int lane, int e);
void tile_word(const TileMap &tm, int i, int *D, int64_t *off);
// Vector copies: when memory positions 0..k-1 (k <= 2) are not register legs
// of the layout, w = 2^k consecutive words of a line sit in w consecutive,
// w-aligned slots, so a lane copies w words at once: copy instruction i
// (i < 2^nreg / w) of lane moves words lane_v + j (j < w) of tile line
// i * w + sub (sub = lane / (32 / w)), i.e. memory tile base + off_v + off_{i*w}
// + j to slots (D_v ^ D_{i*w}) + j, with (D_v, off_v) = tile_vec_lane(lane).
int tile_vec(const TileMap &tm);
void tile_vec_lane(const TileMap &tm, int w, int lane, int *D, int64_t *off);

// Source of the specialised kernel `name` for one chain (exposed for tests).
std::string jit_chain_source(const ChainParams &p, Dtype dt, const std::string &name);

// NVRTC compilation of a generated source to an sm_103a cubin (no device
// needed; exposed for host checks of generated kernels).
bool jit_compile_source(const std::string &src, const std::string &name, std::string *cubin,
                        std::string *err);

// Launch a compiled chain kernel with the interpreting kernel's grid.
cudaError_t launch_jit_chain(const void *kernel, const ChainParams &p, const char *arena,
                             const void *Ax, void *Cx, const Batch &bt, cudaStream_t st);

}  // namespace tn
