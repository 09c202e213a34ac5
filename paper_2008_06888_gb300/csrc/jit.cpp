// jit.cpp -- straight-line register-chain kernels compiled at run time.
//
// The interpreting kernel (k_tchain) reads each table gate's descriptor and
// dispatches on its register legs for every outer index.  Here every large
// chain gets its own kernel: the source below spells out the chain's gates
// on 2^RB named registers, with the outer-index decoding and the register-leg
// offsets as constants.  Tables are built by the same device function as in
// the interpreter and every gate does the same additions and maxima in the
// same order, so the results are bit-identical to the interpreter's (and the
// traceback, which replays chains through the interpreter's tables, sees the
// same values).
#include "jit.h"

#include <dlfcn.h>
#include <nvrtc.h>
#include <sys/stat.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <numeric>
#include <sstream>
#include <thread>

namespace tn {

#include "jit_headers.inc"   // kJitTnInternal, kJitChainDev: header texts for NVRTC

namespace {

// threads per block and resident blocks per SM of a chain with RB register legs
// six-leg chains: TN_JIT_SHAPE6="threads:blocks" overrides the launch shape
std::pair<int, int> shape6() {
  static const std::pair<int, int> sh = [] {
    std::pair<int, int> d{128, 3};
    if (const char *e = std::getenv("TN_JIT_SHAPE6")) {
      int a = 0, b = 0;
      if (std::sscanf(e, "%d:%d", &a, &b) == 2 && a % 32 == 0 && a >= 32 && a <= 256 && b >= 1 &&
          b <= 16)
        d = {a, b};
    }
    return d;
  }();
  return sh;
}
int threads_for(int RB) { return RB >= 6 ? shape6().first : 256; }
int blocks_per_sm(int RB) { return RB >= 6 ? shape6().second : 2; }
size_t smem_for(int RB) { return (size_t)2 * (32 << RB) * (threads_for(RB) / 32) * 4; }

uint64_t fnv1a(const std::string &s, uint64_t h = 1469598103934665603ull) {
  for (unsigned char c : s) {
    h ^= c;
    h *= 1099511628211ull;
  }
  return h;
}

std::string cache_dir() {
  if (const char *d = std::getenv("TN_JIT_CACHE")) return d;
  Dl_info info;
  if (dladdr(reinterpret_cast<const void *>(&fnv1a), &info) && info.dli_fname) {
    std::string f = info.dli_fname;
    const size_t sl = f.rfind('/');
    if (sl != std::string::npos) return f.substr(0, sl) + "/_jit_cache";
  }
  return "";
}

bool read_file(const std::string &path, std::string *out) {
  std::ifstream in(path, std::ios::binary);
  if (!in) return false;
  std::ostringstream ss;
  ss << in.rdbuf();
  *out = ss.str();
  return !out->empty();
}

void write_file_atomic(const std::string &path, const std::string &data) {
  const std::string tmp = path + ".tmp" + std::to_string((unsigned long long)std::hash<std::thread::id>()(std::this_thread::get_id()));
  {
    std::ofstream out(tmp, std::ios::binary);
    if (!out) return;
    out.write(data.data(), (std::streamsize)data.size());
    if (!out) return;
  }
  std::rename(tmp.c_str(), path.c_str());
}

// NVRTC: source -> cubin for sm_103a
bool compile(const std::string &src, const std::string &name, std::string *cubin,
             std::string *err) {
  nvrtcProgram prog;
  const char *hdrs[2] = {kJitTnInternal, kJitChainDev};
  const char *names[2] = {"tn_internal.h", "chain_dev.cuh"};
  if (nvrtcCreateProgram(&prog, src.c_str(), (name + ".cu").c_str(), 2, hdrs, names) !=
      NVRTC_SUCCESS) {
    *err = "nvrtcCreateProgram failed";
    return false;
  }
  const char *opts[] = {"-arch=sm_103a", "-std=c++17", "-default-device", "--ptxas-options=-v"};
  const bool verbose = std::getenv("TN_JIT_VERBOSE") != nullptr;
  const nvrtcResult r = nvrtcCompileProgram(prog, verbose ? 4 : 3, opts);
  if (verbose && r == NVRTC_SUCCESS) {
    size_t n = 0;
    nvrtcGetProgramLogSize(prog, &n);
    std::string log(n, '\0');
    if (n) nvrtcGetProgramLog(prog, &log[0]);
    std::fprintf(stderr, "%s: %s\n", name.c_str(), log.c_str());
  }
  if (r != NVRTC_SUCCESS) {
    size_t n = 0;
    nvrtcGetProgramLogSize(prog, &n);
    std::string log(n, '\0');
    if (n) nvrtcGetProgramLog(prog, &log[0]);
    *err = std::string("nvrtc: ") + nvrtcGetErrorString(r) + "\n" + log;
    nvrtcDestroyProgram(&prog);
    return false;
  }
  size_t n = 0;
  nvrtcGetCUBINSize(prog, &n);
  cubin->assign(n, '\0');
  nvrtcGetCUBIN(prog, &(*cubin)[0]);
  nvrtcDestroyProgram(&prog);
  return n > 0;
}

struct Loaded {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kernel = nullptr;
};

std::mutex g_mu;
std::map<std::pair<int, uint64_t>, Loaded> g_loaded;   // (device, source hash)

bool worth(const ChainParams &p) {
  static const long long min_el = [] {
    const char *s = std::getenv("TN_JIT_MIN_ELEMENTS");
    return s ? std::atoll(s) : (1ll << 15);
  }();
  return p.mode == 1 && p.P == 0 && (p.t == 5 || p.t == 6) && p.ntg > 0 &&
         p.outer * p.tile >= min_el;
}

}  // namespace

bool tile_map(const ChainParams &p, const int64_t *hi, TileMap *tm) {
  const int RB = p.t;
  if (p.mode != 1 || RB < 5 || RB > 6 || p.outer % 32) return false;
  *tm = TileMap{};
  int regpos[6];
  for (int b = 0; b < RB; ++b) {
    if (hi[1 << b] == 0) continue;   // not a leg of this layout
    int q = 0;
    while ((int64_t(1) << q) < hi[1 << b]) ++q;
    tm->rbit[tm->nreg] = b;
    regpos[tm->nreg++] = q;
  }
  auto reg_of = [&](int pos) {
    for (int k = 0; k < tm->nreg; ++k)
      if (regpos[k] == pos) return k;
    return -1;
  };
  // one low leg by default: two (16-byte owner accesses) measured the same
  // and spill a few registers in some chains
  static const int low_max = std::getenv("TN_JIT_NO_LOW_LEGS") ? 0
                             : std::getenv("TN_JIT_LOW_MAX")   ? std::atoi(std::getenv("TN_JIT_LOW_MAX"))
                                                               : 1;
  int a = 0;
  while (a < low_max && a < 2 && reg_of(a) >= 0) ++a;
  tm->a = a;
  int m = 0;
  for (int q = 0; q < 5; ++q) m += reg_of(q) < 0;
  int k = 0;
  for (int q = a; q < 5; ++q)
    if (reg_of(q) >= 0) tm->gbit[reg_of(q)] = 1 << (m + k++);
  int nh = 0;
  for (int c = 0; c < tm->nreg; ++c) {
    tm->lowbit[c] = regpos[c] < a ? regpos[c] : -1;
    tm->hibit[c] = regpos[c] < a ? -1 : nh++;
  }
  int rank = 0;
  for (int q = 0; (int)tm->tpos.size() < 5 + tm->nreg && q < 62; ++q) {
    const int c = reg_of(q);
    if (c >= 0) {
      tm->tpos.push_back(q);
      tm->cbit.push_back(tm->lowbit[c] >= 0 ? 1 << tm->lowbit[c]
                                            : (1 << (5 + a + tm->hibit[c])) ^ (tm->gbit[c] << a));
    } else if (rank++ < 5) {
      tm->tpos.push_back(q);
      tm->cbit.push_back(1 << (a + rank - 1));
    }
  }
  if ((int)tm->tpos.size() != 5 + tm->nreg) return false;
  for (int j = 0; j < 5; ++j)
    if (tm->tpos[j] != j) return false;   // positions 0..4 are always tile bits
  return true;
}

int tile_slot(const TileMap &tm, int lane, int e) {
  int c = 0, g = 0, low = 0;
  for (int k = 0; k < tm.nreg; ++k)
    if ((e >> tm.rbit[k]) & 1) {
      if (tm.lowbit[k] >= 0) {
        low |= 1 << tm.lowbit[k];
      } else {
        c |= 1 << tm.hibit[k];
        g ^= tm.gbit[k];
      }
    }
  return (c << (5 + tm.a)) | ((lane ^ g) << tm.a) | low;
}

void tile_word(const TileMap &tm, int i, int *D, int64_t *off) {
  *D = 0;
  *off = 0;
  for (int k = 0; k < tm.nreg; ++k)
    if ((i >> k) & 1) {
      *D ^= tm.cbit[5 + k];
      *off += int64_t(1) << tm.tpos[5 + k];
    }
}

int tile_vec(const TileMap &tm) {
  int k = 0;
  while (k < 2 && tm.cbit[k] == (1 << k)) ++k;
  while ((1 << k) > (1 << tm.nreg)) --k;   // a copy instruction spans w tile lines
  return 1 << k;
}

void tile_vec_lane(const TileMap &tm, int w, int lane, int *D, int64_t *off) {
  const int per = 32 / w, sub = lane / per, first = (lane % per) * w;
  *D = 0;
  *off = first;
  for (int j = 0; j < 5; ++j)
    if ((first >> j) & 1) *D ^= tm.cbit[j];
  for (int k = 0; (1 << k) < w; ++k)
    if ((sub >> k) & 1) {
      *D ^= tm.cbit[5 + k];
      *off += int64_t(1) << tm.tpos[5 + k];
    }
}

bool jit_compile_source(const std::string &src, const std::string &name, std::string *cubin,
                        std::string *err) {
  return compile(src, name, cubin, err);
}

std::string jit_chain_source(const ChainParams &p, Dtype dt, const std::string &name) {
  const bool f32 = dt == DT_F32;
  const char *T = f32 ? "float" : "int";
  const char *MX = f32 ? "fmaxf" : "max";
  const int RB = p.t, NT = threads_for(RB);
  const int E = 1 << RB, S = E * NT, W = 32 * E;   // states, slot and warp tile (values)
  TileMap tin, tout;
  if (!tile_map(p, p.hi_in, &tin) || !tile_map(p, p.hi_out, &tout)) return "";
  const bool con = p.ntg > 0 && p.tg[p.ntg - 1].kind == 2;   // final contraction
  const int nmain = con ? p.ntg - 1 : p.ntg;
  const int cmask = con ? 1 << p.tg[p.ntg - 1].J : 0;
  const bool i32 = p.outer * p.tile < (int64_t(1) << 31);
  std::ostringstream o;
  o << "#include \"chain_dev.cuh\"\n"
    << "typedef unsigned long long U;   // two FP32 values\n"
    << "__device__ __forceinline__ U pk2(float a, float b) { U r; asm(\"mov.b64 %0, {%1, %2};\" : \"=l\"(r) : \"f\"(a), \"f\"(b)); return r; }\n"
    << "__device__ __forceinline__ float lo2(U x) { float a, b; asm(\"mov.b64 {%0, %1}, %2;\" : \"=f\"(a), \"=f\"(b) : \"l\"(x)); return a; }\n"
    << "__device__ __forceinline__ float hi2(U x) { float a, b; asm(\"mov.b64 {%0, %1}, %2;\" : \"=f\"(a), \"=f\"(b) : \"l\"(x)); return b; }\n"
    << "__device__ __forceinline__ U add2(U a, U b) { U r; asm(\"add.rn.f32x2 %0, %1, %2;\" : \"=l\"(r) : \"l\"(a), \"l\"(b)); return r; }\n"
    << "extern \"C\" __global__ void __launch_bounds__(" << NT << ", " << blocks_per_sm(RB) << ")\n"
    << name << "(const ChainParams p, const " << T << " *__restrict__ X, const " << T
    << " *__restrict__ A, " << T << " *__restrict__ C, long long ib) {\n"
    << "  using namespace tn;\n"
    << "  typedef " << T << " T;\n"
    << "  typedef " << (i32 ? "int" : "long long") << " I;\n"
    << "  typedef Vec4<T>::t V;\n"
    << "  X = inst_ptr(X, ib);\n  A = inst_ptr(A, ib);\n  C = inst_ptr(C, ib);\n"
    << "  __shared__ __align__(16) T sT[" << std::max(8, (int)p.ttotal) << "];\n"
    << "  extern __shared__ __align__(16) char rstage[];\n"
    << "  T *stage = reinterpret_cast<T *>(rstage);\n"
    << "  const int tid = threadIdx.x, lane = tid & 31;\n"
    << "  const long long step = (long long)gridDim.x * " << NT << ";\n"
    << "  long long tau = blockIdx.x * " << NT << "LL + tid;\n";
  // outer index -> element offset in the input and in the output (segments
  // slowest first)
  for (int side = 0; side < 2; ++side) {
    const int32_t *ssh = side == 0 ? p.ssh_in : p.ssh_out;
    o << "  auto base_" << (side == 0 ? "in" : "out") << " = [](long long t) -> I {\n"
      << "    I b = 0, u = (I)t;\n";
    for (int sg = p.nseg - 1; sg >= 0; --sg)
      o << "    b += (u & (I)" << (p.seg_size[sg] - 1) << ") << " << ssh[sg] << ";\n"
        << "    u >>= " << p.seg_sh[sg] << ";\n";
    o << "    return b;\n  };\n";
  }
  // Tile of a warp: its 32 outer indices x the register states of a layout.
  // Its index bits (word w, memory order) always include memory positions
  // 0..4, so word w = lane + 32 i lies at tile base + lane + off_i: lane
  // copies words lane + 32 i and every copy of the warp moves 128 contiguous
  // bytes.  In the warp's shared-memory tile, register state e of the thread
  // of lane sits at a slot swizzled so that the copies and the owner's reads
  // and writes are free of bank conflicts (TileMap).  Only the warp itself
  // touches its tile (__syncwarp).
  // Vector copies (tile_vec): lane-dependent slot and memory offsets of the
  // first word a lane moves, as in tile_vec_lane.
  const bool vec = std::getenv("TN_JIT_NO_VEC") == nullptr;
  const int win = vec ? tile_vec(tin) : 1, wout = vec ? tile_vec(tout) : 1;
  // 16-byte copies bypass L1 (.cg) unless the layout has low register legs:
  // there the two lanes that share a 32-byte sector write shared-memory slots
  // that are apart, and a bypassing copy reads the sector once per lane
  static const char *ca_env = std::getenv("TN_JIT_CA16");   // "0": never, "1": always
  const bool ca16 = ca_env ? *ca_env == '1' : tin.a > 0;
  auto lane_vec = [&](const TileMap &tm, int w, const char *Dn, const char *On) {
    std::ostringstream d;
    const int per = 32 / w;
    d << "  const int " << Dn << " = 0";
    for (int j = 0; j < 5; ++j)
      d << " ^ (-((((lane % " << per << ") * " << w << ") >> " << j << ") & 1) & " << tm.cbit[j] << ")";
    for (int k = 0; (1 << k) < w; ++k)
      d << " ^ (-(((lane / " << per << ") >> " << k << ") & 1) & " << tm.cbit[5 + k] << ")";
    d << ";\n  const int " << On << " = (lane % " << per << ") * " << w;
    for (int k = 0; (1 << k) < w; ++k)
      d << " + ((((lane / " << per << ") >> " << k << ") & 1) << " << tm.tpos[5 + k] << ")";
    d << ";\n";
    return d.str();
  };
  o << "  T *const wstage = stage + (tid >> 5) * " << W << ";\n"
    << lane_vec(tin, win, "Din", "Oin") << lane_vec(tout, wout, "Dout", "Oout")
    << "  auto issue = [&](long long t, int s) {\n"
    << "    if (t < " << p.outer << "LL) {\n"
    << "      const T *src = A + base_in(t - lane) + Oin;\n"
    << "      T *dst = wstage + s * " << S << ";\n";
  for (int i = 0; i < (1 << tin.nreg); i += win) {
    int D;
    int64_t off;
    tile_word(tin, i, &D, &off);
    o << "      cp_async" << 4 * win << (win == 4 && ca16 ? "ca" : "") << "(dst + (Din ^ " << D
      << "), src + " << off << ");\n";
  }
  o << "    }\n    cp_async_commit();\n  };\n"
    << "  issue(tau, 0);\n"
    << "  build_tables<T>(p, X, sT);\n"
    << "  __syncthreads();\n"
    << "  for (int it = 0; tau < " << p.outer << "LL; tau += step, ++it) {\n"
    << "    const int cur = it & 1;\n"
    << "    issue(tau + step, cur ^ 1);\n"
    << "    cp_async_wait_prev();\n"
    << "    __syncwarp();\n"   // words of the tile come from other lanes
    << "    T *const sw = wstage + cur * " << S << ";\n";
  auto gate_table = [&](const TGate &t, std::ostringstream &g) {
    std::ostringstream f;
    if (t.nf == 0) f << "0";
    for (int i = 0; i < t.nf; ++i) {
      if (i) f << " | ";
      f << "((int)((tau >> " << (int)t.fsh[i] << ") & 1) << " << i << ")";
    }
    g << "      const int f = " << f.str() << ";\n"
      << "      const V lo = *reinterpret_cast<const V *>(sT + " << t.toff << " + f * 8);\n";
    if (t.kind != 1 && t.K >= 0)
      g << "      const V hi = *reinterpret_cast<const V *>(sT + " << t.toff << " + f * 8 + 4);\n";
  };
  // FP32 chains keep their states in pairs (state e with bit P clear, and e | P)
  // in 64-bit registers: a replace gate on another bit then does the adds of two
  // state pairs with two-wide FP32 adds (add.rn.f32x2: each lane rounds like a
  // scalar add, so results are unchanged) and the maxima on the halves.  P is the
  // register leg with the fewest replace gates.
  int P = -1;
  if (f32 && std::getenv("TN_JIT_NO_F32X2") == nullptr) {
    int cnt[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 0; k < p.ntg; ++k)
      if (p.tg[k].kind != 1) cnt[p.tg[k].J]++;
    // cost of a packing leg: a replace gate on it runs on the halves (about
    // 64 more instructions than on a packed pair), and a layout whose first
    // low leg is another leg needs register moves to pair the states of its
    // vector accesses (about 64 per side)
    auto low0 = [](const TileMap &tm) {
      for (int k = 0; k < tm.nreg; ++k)
        if (tm.lowbit[k] == 0) return tm.rbit[k];
      return -1;
    };
    static const bool by_gates = std::getenv("TN_JIT_P_BY_GATES") != nullptr;
    const int l_in = by_gates ? -1 : low0(tin), l_out = by_gates ? -1 : low0(tout);
    auto cost = [&](int b) {
      return 64 * cnt[b] + (l_in >= 0 && l_in != b ? 64 : 0) + (l_out >= 0 && l_out != b ? 64 : 0);
    };
    P = 0;
    for (int b = 1; b < RB; ++b)
      if (cost(b) <= cost(P)) P = b;
  }
  // Register states from the input tile: one access per group of the 2^a
  // states that differ in the low legs (a vector of 2^a words); a state of a
  // leg the input layout lacks (a rank-raising chain) reads its source state.
  auto vec_type = [](int a) {
    return a == 2 ? std::string("V") : a == 1 ? std::string("typename Vec2<T>::t") : std::string("T");
  };
  auto slot_expr = [](const TileMap &tm, int sl) {
    // tile_slot(tm, lane, e) with sl = tile_slot(tm, 0, e) and its low bits cleared
    std::ostringstream x;
    x << "sw + " << (sl & ~((32 << tm.a) - 1)) << " + ((lane ^ " << ((sl >> tm.a) & 31) << ") << "
      << tm.a << ")";
    return x.str();
  };
  static const char *kComp[4] = {".x", ".y", ".z", ".w"};
  std::map<int, int> in_group;   // slot of low bits 0 -> load index
  std::vector<std::string> in_val(E);
  for (int e = 0; e < E; ++e) {
    const int sl = tile_slot(tin, 0, e), key = sl & ~((1 << tin.a) - 1);
    auto it = in_group.find(key);
    if (it == in_group.end()) {
      it = in_group.emplace(key, (int)in_group.size()).first;
      o << "    const " << vec_type(tin.a) << " r" << it->second << " = *reinterpret_cast<const "
        << vec_type(tin.a) << " *>(" << slot_expr(tin, key) << ");\n";
    }
    in_val[e] = "r" + std::to_string(it->second) + (tin.a ? kComp[sl & ((1 << tin.a) - 1)] : "");
  }
  if (P < 0) {
    for (int e = 0; e < E; ++e) o << "    T v" << e << " = " << in_val[e] << ";\n";
    o << "    __syncwarp();\n";   // the slot is reused for the outputs below
    for (int k = 0; k < p.ntg; ++k) {
      const TGate &t = p.tg[k];
      std::ostringstream g;
      g << "    {  // table gate " << k
        << (t.kind == 0 ? ": replace" : t.kind == 2 ? ": final contraction" : ": diagonal") << "\n";
      gate_table(t, g);
      if (t.kind == 0 || t.kind == 2) {
        for (int e = 0; e < E; ++e) {
          if (e & (1 << t.J)) continue;
          const int e1 = e | (1 << t.J);
          const char *tb = (t.K >= 0 && ((e >> t.K) & 1)) ? "hi" : "lo";
          if (t.kind == 0)
            g << "      { const T a = v" << e << ", b = v" << e1 << "; v" << e << " = " << MX << "(a + "
              << tb << ".x, b + " << tb << ".y); v" << e1 << " = " << MX << "(a + " << tb
              << ".z, b + " << tb << ".w); }\n";
          else
            g << "      v" << e << " = " << MX << "(v" << e << " + " << tb << ".x, v" << e1 << " + "
              << tb << ".y);\n";
        }
      } else {
        for (int e = 0; e < E; ++e) {
          const int x0 = t.J >= 0 ? (e >> t.J) & 1 : 0, x1 = t.K >= 0 ? (e >> t.K) & 1 : 0;
          const char *c = x1 ? (x0 ? "w" : "z") : (x0 ? "y" : "x");
          g << "      v" << e << " = v" << e << " + lo." << c << ";\n";
        }
      }
      g << "    }\n";
      o << g.str();
    }
  } else {
    const int PM = 1 << P;
    for (int e = 0; e < E; ++e)
      if (!(e & PM)) o << "    U u" << e << " = pk2(" << in_val[e] << ", " << in_val[e | PM] << ");\n";
    o << "    __syncwarp();\n";   // the slot is reused for the outputs below
    auto tabsel = [](int k, int kdig) { return kdig ? "hi" : "lo"; };
    for (int k = 0; k < p.ntg; ++k) {
      const TGate &t = p.tg[k];
      std::ostringstream g;
      g << "    {  // table gate " << k
        << (t.kind == 0 ? ": replace" : t.kind == 2 ? ": final contraction" : ": diagonal") << "\n";
      gate_table(t, g);
      const char *comp[4] = {"x", "y", "z", "w"};
      if (t.kind != 1 && t.J == P) {
        // the gate's own pairs are the two halves of one register
        for (int e = 0; e < E; ++e) {
          if (e & PM) continue;
          const char *tb = tabsel(k, t.K >= 0 && ((e >> t.K) & 1));
          if (t.kind == 0)
            g << "      { const float a = lo2(u" << e << "), b = hi2(u" << e << "); u" << e
              << " = pk2(fmaxf(a + " << tb << ".x, b + " << tb << ".y), fmaxf(a + " << tb
              << ".z, b + " << tb << ".w)); }\n";
          else
            g << "      { const float a = lo2(u" << e << "), b = hi2(u" << e << "); u" << e
              << " = pk2(fmaxf(a + " << tb << ".x, b + " << tb << ".y), 0.f); }\n";
        }
      } else if (t.kind != 1) {
        // packed table constants: the P half may read the other K table
        const int nsets = (t.K >= 0 && t.K != P) ? 2 : 1;
        for (int set = 0; set < nsets; ++set)
          for (int c = 0; c < (t.kind == 0 ? 4 : 2); ++c) {
            const char *lt = t.K == P ? "lo" : tabsel(k, set);
            const char *ht = t.K == P ? "hi" : tabsel(k, set);
            g << "      const U T" << set << c << " = pk2(" << lt << "." << comp[c] << ", " << ht << "."
              << comp[c] << ");\n";
          }
        for (int e = 0; e < E; ++e) {
          if ((e & PM) || (e & (1 << t.J))) continue;
          const int e1 = e | (1 << t.J);
          const int set = (t.K >= 0 && t.K != P) ? ((e >> t.K) & 1) : 0;
          if (t.kind == 0)
            g << "      { const U x0 = add2(u" << e << ", T" << set << "0), y0 = add2(u" << e1 << ", T"
              << set << "1), x1 = add2(u" << e << ", T" << set << "2), y1 = add2(u" << e1 << ", T" << set
              << "3); u" << e << " = pk2(fmaxf(lo2(x0), lo2(y0)), fmaxf(hi2(x0), hi2(y0))); u" << e1
              << " = pk2(fmaxf(lo2(x1), lo2(y1)), fmaxf(hi2(x1), hi2(y1))); }\n";
          else
            g << "      { const U x0 = add2(u" << e << ", T" << set << "0), y0 = add2(u" << e1 << ", T"
              << set << "1); u" << e << " = pk2(fmaxf(lo2(x0), lo2(y0)), fmaxf(hi2(x0), hi2(y0))); }\n";
        }
      } else {
        for (int e = 0; e < E; ++e) {
          if (e & PM) continue;
          auto cval = [&](int st) {
            const int x0 = t.J >= 0 ? (st >> t.J) & 1 : 0, x1 = t.K >= 0 ? (st >> t.K) & 1 : 0;
            return std::string("lo.") + (x1 ? (x0 ? "w" : "z") : (x0 ? "y" : "x"));
          };
          g << "      u" << e << " = add2(u" << e << ", pk2(" << cval(e) << ", " << cval(e | PM) << "));\n";
        }
      }
      g << "    }\n";
      o << g.str();
    }
    // unpack for the stores below
    for (int e = 0; e < E; ++e) {
      if (e & cmask) continue;
      o << "    const T v" << e << " = " << ((e & PM) ? "hi2(u" : "lo2(u") << (e & ~PM) << ");\n";
    }
  }
  (void)nmain;
  // outputs through the warp's tile, then whole 128-byte lines
  // every group of 2^a output states fills one vector (the output layout has
  // every leg but a contracted one)
  std::map<int, std::vector<int>> out_group;
  for (int e = 0; e < E; ++e) {
    if (e & cmask) continue;
    const int sl = tile_slot(tout, 0, e), key = sl & ~((1 << tout.a) - 1);
    auto &gv = out_group[key];
    gv.resize(1 << tout.a, -1);
    if (gv[sl & ((1 << tout.a) - 1)] != -1) return "";
    gv[sl & ((1 << tout.a) - 1)] = e;
  }
  for (auto &kv : out_group) {
    o << "    *reinterpret_cast<" << vec_type(tout.a) << " *>(" << slot_expr(tout, kv.first) << ") = ";
    if (tout.a) o << vec_type(tout.a) << "{";
    for (size_t j = 0; j < kv.second.size(); ++j) {
      if (kv.second[j] < 0) return "";
      o << (j ? ", " : "") << "v" << kv.second[j];
    }
    o << (tout.a ? "};\n" : ";\n");
  }
  o << "    __syncwarp();\n"
    << "    T *dst = C + base_out(tau - lane) + Oout;\n";
  const char *VT = wout == 4 ? "V" : wout == 2 ? "typename Vec2<T>::t" : "T";
  for (int i = 0; i < (1 << tout.nreg); i += wout) {
    int D;
    int64_t off;
    tile_word(tout, i, &D, &off);
    o << "    *reinterpret_cast<" << VT << " *>(dst + " << off << ") = *reinterpret_cast<const "
      << VT << " *>(sw + (Dout ^ " << D << "));\n";
  }
  o << "    __syncwarp();\n"   // the tile is refilled by a later issue
    << "  }\n  asm volatile(\"cp.async.wait_all;\\n\" ::: \"memory\");\n}\n";
  return o.str();
}

bool jit_chains(const std::vector<ChainParams> &chains, Dtype dt, std::vector<const void *> *out,
                std::string *err) {
  out->assign(chains.size(), nullptr);
  if (std::getenv("TN_NO_JIT")) return true;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    *err = "no CUDA device for the chain kernels";
    return false;
  }
  int nvrtc_major = 0, nvrtc_minor = 0;
  nvrtcVersion(&nvrtc_major, &nvrtc_minor);
  const std::string tag = "sm_103a nvrtc " + std::to_string(nvrtc_major) + "." +
                          std::to_string(nvrtc_minor) + "\n";
  struct Job {
    size_t idx;
    uint64_t h;
    std::string name, src, cubin, err;
    bool ok = false;
  };
  std::vector<Job> jobs;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (size_t i = 0; i < chains.size(); ++i) {
      if (!worth(chains[i])) continue;
      Job j;
      j.idx = i;
      const std::string probe = jit_chain_source(chains[i], dt, "tn_chain");
      if (probe.empty()) continue;   // no tile map: the chain stays interpreted
      j.h = fnv1a(tag + probe);
      char nm[40];
      std::snprintf(nm, sizeof(nm), "tn_chain_%016llx", (unsigned long long)j.h);
      j.name = nm;
      auto it = g_loaded.find({dev, j.h});
      if (it != g_loaded.end()) {
        (*out)[i] = reinterpret_cast<const void *>(it->second.kernel);
        continue;
      }
      j.src = jit_chain_source(chains[i], dt, j.name);
      jobs.push_back(std::move(j));
    }
  }
  if (jobs.empty()) return true;
  const std::string dir = cache_dir();
  if (!dir.empty()) mkdir(dir.c_str(), 0755);
  std::atomic<size_t> next{0};
  auto work = [&]() {
    for (size_t k; (k = next.fetch_add(1)) < jobs.size();) {
      Job &j = jobs[k];
      const std::string path = dir.empty() ? "" : dir + "/" + j.name + ".cubin";
      if (!path.empty() && read_file(path, &j.cubin)) {
        j.ok = true;
        continue;
      }
      j.ok = compile(j.src, j.name, &j.cubin, &j.err);
      if (j.ok && !path.empty()) write_file_atomic(path, j.cubin);
    }
  };
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t nth = std::min<size_t>(jobs.size(), std::min(32u, hw));
  std::vector<std::thread> pool;
  for (size_t t = 1; t < nth; ++t) pool.emplace_back(work);
  work();
  for (auto &t : pool) t.join();
  std::lock_guard<std::mutex> lk(g_mu);
  for (Job &j : jobs) {
    const size_t smem = smem_for(chains[j.idx].t);
    if (!j.ok) {
      *err = "chain kernel " + j.name + ": " + j.err;
      return false;
    }
    auto it = g_loaded.find({dev, j.h});
    if (it == g_loaded.end()) {
      Loaded L;
      cudaError_t e = cudaLibraryLoadData(&L.lib, j.cubin.data(), nullptr, nullptr, 0, nullptr,
                                          nullptr, 0);
      if (e == cudaSuccess) e = cudaLibraryGetKernel(&L.kernel, L.lib, j.name.c_str());
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(reinterpret_cast<const void *>(L.kernel),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) {
        cudaGetLastError();
        *err = "loading chain kernel " + j.name + ": " + cudaGetErrorString(e);
        return false;
      }
      it = g_loaded.emplace(std::make_pair(dev, j.h), L).first;
    }
    (*out)[j.idx] = reinterpret_cast<const void *>(it->second.kernel);
  }
  return true;
}

// SMs of the current device (this file also builds into host-only checks,
// without kernels.cu)
static int jit_sms() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
    return 152;
  return v;
}

cudaError_t launch_jit_chain(const void *kernel, const ChainParams &p, const char *arena,
                             const void *Ax, void *Cx, const Batch &bt, cudaStream_t st) {
  if (p.outer == 0) return cudaSuccess;
  const int NT = threads_for(p.t);
  const int64_t need = (p.outer + NT - 1) / NT;
  // blocks per instance: the B instances' blocks should fill the resident
  // slots (SMs x blocks per SM) in whole waves, so that every SM carries the
  // same number of equal blocks; else one partial wave
  const int64_t slots = (int64_t)jit_sms() * blocks_per_sm(p.t);
  const int64_t cap = std::max<int64_t>(1, slots / bt.B);
  const int64_t whole = slots / std::gcd(slots, (int64_t)bt.B);
  int64_t blocks = std::min(need, cap);
  if (whole <= need && whole <= 4 * cap) blocks = whole;
  // the compiled tile copies move up to 16 bytes per lane
  if ((reinterpret_cast<uintptr_t>(Ax) | reinterpret_cast<uintptr_t>(Cx) | (uintptr_t)bt.ib) & 15)
    return cudaErrorMisalignedAddress;
  ChainParams pc = p;
  const void *X = arena;
  const void *A = Ax;
  void *C = Cx;
  long long ib = bt.ib;
  void *args[] = {&pc, &X, &A, &C, &ib};
  return cudaLaunchKernel(kernel, dim3((unsigned)blocks, bt.B), dim3(NT), args, smem_for(p.t), st);
}

}  // namespace tn
