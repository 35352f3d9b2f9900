// Class-specialised step and adjoint kernels compiled at run time (NVRTC).
//
// A class-constant launch (one class, propellers, Euler, hover task) reads
// its class tables as constant-bank operands: the arithmetic cannot know that
// half of the allocation matrix is zero (each propeller of the workload
// layouts drives three of the six wrench rows), that the centre of buoyancy
// lies on the body z axis, or that a neutral vehicle has W = B. Compiled with
// the class's values as literals, those terms fold away. This file builds
// such kernels from the library's own kernel headers (embedded at build
// time): one NVRTC program per (device architecture, kernel, thruster count,
// single- or multi-step launch, class table), compiled to a cubin for the
// device and loaded as a CUDA library; compiled kernels are kept for the
// process. The adjoint kernel takes only the actuator tables as literals
// (its physical parameters are per env). NVRTC is loaded with dlopen:
// without it (or if a compile fails) the launches keep the kernels built
// with the library.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "mg_internal.h"
#include "mg_jit_sources.inc"   // kJitHeaderNames / kJitHeaderBodies (generated by the build)

#ifndef MG_USE_PDL
#define MG_USE_PDL 1
#endif

namespace mg {

size_t step_kernel_smem_jit(int nt, int pm);

namespace {

struct Nvrtc {
  bool ok = false;
  nvrtcResult (*create)(nvrtcProgram*, const char*, const char*, int, const char* const*, const char* const*);
  nvrtcResult (*destroy)(nvrtcProgram*);
  nvrtcResult (*compile)(nvrtcProgram, int, const char* const*);
  nvrtcResult (*log_size)(nvrtcProgram, size_t*);
  nvrtcResult (*log)(nvrtcProgram, char*);
  nvrtcResult (*add_name)(nvrtcProgram, const char*);
  nvrtcResult (*lowered)(nvrtcProgram, const char*, const char**);
  nvrtcResult (*cubin_size)(nvrtcProgram, size_t*);
  nvrtcResult (*cubin)(nvrtcProgram, char*);
};

const Nvrtc& nvrtc() {
  static Nvrtc n = [] {
    Nvrtc r;
    void* h = nullptr;
    for (const char* name : {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"}) {
      h = dlopen(name, RTLD_NOW | RTLD_LOCAL);
      if (h) break;
    }
    if (!h) return r;
    auto sym = [&](const char* s) { return dlsym(h, s); };
    r.create = reinterpret_cast<decltype(r.create)>(sym("nvrtcCreateProgram"));
    r.destroy = reinterpret_cast<decltype(r.destroy)>(sym("nvrtcDestroyProgram"));
    r.compile = reinterpret_cast<decltype(r.compile)>(sym("nvrtcCompileProgram"));
    r.log_size = reinterpret_cast<decltype(r.log_size)>(sym("nvrtcGetProgramLogSize"));
    r.log = reinterpret_cast<decltype(r.log)>(sym("nvrtcGetProgramLog"));
    r.add_name = reinterpret_cast<decltype(r.add_name)>(sym("nvrtcAddNameExpression"));
    r.lowered = reinterpret_cast<decltype(r.lowered)>(sym("nvrtcGetLoweredName"));
    r.cubin_size = reinterpret_cast<decltype(r.cubin_size)>(sym("nvrtcGetCUBINSize"));
    r.cubin = reinterpret_cast<decltype(r.cubin)>(sym("nvrtcGetCUBIN"));
    r.ok = r.create && r.destroy && r.compile && r.log_size && r.log && r.add_name && r.lowered && r.cubin_size &&
           r.cubin;
    return r;
  }();
  return n;
}

struct Entry {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kern = nullptr;
  bool failed = false;
  std::string err;
};

std::mutex g_mu;
std::map<std::string, Entry> g_cache;

// A float as an exact C++ literal.
std::string lit(float v) {
  char b[64];
  if (v == 0.0f) return std::signbit(v) ? "-0.0f" : "0.0f";
  std::snprintf(b, sizeof(b), "%af", (double)v);
  return b;
}

std::string class_source(const ClassK& k, const char* header) {
  std::string s = std::string("#include \"") + header +
                  "\"\nnamespace mg {\nstruct JitLit {\n  MG_HD static constexpr ClassK make() {\n    ClassK k{};\n";
  auto arr = [&](const char* name, const float* v, int n) {
    for (int i = 0; i < n; ++i) s += std::string("    k.") + name + "[" + std::to_string(i) + "] = " + lit(v[i]) + ";\n";
  };
  for (int r = 0; r < 6; ++r)
    for (int i = 0; i < 8; ++i)
      s += "    k.alloc[" + std::to_string(r) + "][" + std::to_string(i) + "] = " + lit(k.alloc[r][i]) + ";\n";
  arr("kf", k.kf, 8);
  arr("dz", k.dz, 8);
  arr("alpha", k.alpha, 8);
  arr("minv", k.minv, 6);
  arr("A", k.A, 6);
  arr("dl", k.dl, 6);
  arr("dq", k.dq, 6);
  s += "    k.m = " + lit(k.m) + ";\n";
  arr("Ig", k.Ig, 3);
  s += "    k.W = " + lit(k.W) + ";\n    k.B = " + lit(k.B) + ";\n";
  arr("rb", k.rb, 3);
  arr("Vc", k.Vc, 3);
  s += "    k.dz_on = " + std::to_string(k.dz_on) + "u;\n    return k;\n  }\n};\n}  // namespace mg\n";
  return s;
}

enum Kind { STEP = 0, ADJOINT = 1 };

std::string kernel_name(Kind kind, int nt, bool ms, int pm) {
  if (kind == ADJOINT) return "mg::mg_adjoint_kernel<" + std::to_string(nt) + ", false, mg::JitLit>";
  return "mg::mg_step_kernel<" + std::to_string(nt) + ", " + std::to_string(pm) + ", 0, true, false, " +
         (ms ? "true" : "false") + ", mg::JitLit>";
}

// Compile and load one specialised kernel (caller holds g_mu). Step kernels
// are compiled for min_blocks resident blocks per SM (their launch bounds).
void build(Entry& e, Kind kind, const ClassK& k, int nt, bool ms, int pm, int arch, int min_blocks) {
  const Nvrtc& n = nvrtc();
  if (!n.ok) { e.failed = true; e.err = "NVRTC not available"; return; }
  const std::string src = class_source(k, kind == ADJOINT ? "mg_adjoint.cuh" : "mg_step.cuh");
  nvrtcProgram prog = nullptr;
  if (n.create(&prog, src.c_str(), "mg_jit_step.cu", kJitHeaderCount, kJitHeaderBodies, kJitHeaderNames) !=
      NVRTC_SUCCESS) {
    e.failed = true; e.err = "nvrtcCreateProgram failed"; return;
  }
  const std::string name = kernel_name(kind, nt, ms, pm);
  n.add_name(prog, name.c_str());
  const std::string arch_opt = "--gpu-architecture=sm_" + std::to_string(arch) + "a";
  const std::string blocks_opt = "-DMG_KSTEP_MIN_BLOCKS=" + std::to_string(min_blocks);
  // Step kernels alias each warp's observation tile into its stage buffer
  // (a sixth block of every thruster count then fits an SM's shared memory).
  const char* opts[] = {arch_opt.c_str(), "-std=c++17", "-default-device", "-lineinfo", blocks_opt.c_str(),
                        "-DMG_OBS_ALIAS=1"};
  const nvrtcResult rc = n.compile(prog, kind == ADJOINT ? 4 : 6, opts);
  if (rc != NVRTC_SUCCESS) {
    size_t ls = 0;
    n.log_size(prog, &ls);
    std::string lg(ls, '\0');
    if (ls) n.log(prog, &lg[0]);
    e.failed = true;
    e.err = "NVRTC compile failed: " + lg.substr(0, 400);
    n.destroy(&prog);
    return;
  }
  const char* low = nullptr;
  size_t cs = 0;
  n.lowered(prog, name.c_str(), &low);
  n.cubin_size(prog, &cs);
  std::vector<char> cubin(cs);
  if (cs) n.cubin(prog, cubin.data());
  const std::string lowered = low ? low : "";
  n.destroy(&prog);
  if (lowered.empty() || cubin.empty()) { e.failed = true; e.err = "NVRTC produced no kernel"; return; }
  if (cudaLibraryLoadData(&e.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess ||
      cudaLibraryGetKernel(&e.kern, e.lib, lowered.c_str()) != cudaSuccess) {
    cudaGetLastError();
    e.failed = true;
    e.err = "loading the compiled kernel failed";
    e.kern = nullptr;
    return;
  }
  if (kind == ADJOINT) return;   // static shared memory only
  const int smem = (int)step_kernel_smem_jit(nt, pm);
  if (cudaFuncSetAttribute(reinterpret_cast<const void*>(e.kern), cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
      cudaSuccess) {
    cudaGetLastError();
    e.failed = true;
    e.err = "setting the kernel's shared memory failed";
    e.kern = nullptr;
  }
}

const void* jit_kernel(Kind kind, const ClassK& k, int nt, bool ms, int pm, int min_blocks, std::string* err) {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) !=
                                                cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
    cudaGetLastError();
    if (err) *err = "no device";
    return nullptr;
  }
  const int arch = major * 10 + minor;
  std::string key(reinterpret_cast<const char*>(&k), sizeof(k));
  key += ":" + std::to_string((int)kind) + ":" + std::to_string(dev) + ":" + std::to_string(arch) + ":" +
         std::to_string(nt) + (ms ? ":ms" : ":1") + ":" + std::to_string(min_blocks) + ":pm" + std::to_string(pm);
  std::lock_guard<std::mutex> lk(g_mu);
  Entry& e = g_cache[key];
  if (!e.kern && !e.failed) build(e, kind, k, nt, ms, pm, arch, min_blocks);
  if (e.failed) {
    if (err) *err = e.err;
    return nullptr;
  }
  return reinterpret_cast<const void*>(e.kern);
}

}  // namespace

// Resident blocks per SM that the class-specialised step kernel of a launch
// of n_tiles tiles at K substeps is compiled for. The literal class tables
// bring these kernels to 80 registers at a bound of 6 blocks per SM (105-114
// at 4, the bound of the library's kernels), without spills, and with each
// warp's observation tile aliased into its stage buffer six blocks of every
// thruster count fit an SM's shared memory: more warps hide more of the
// substep's dependency latency, but the persistent grid's blocks walk fewer
// tiles. Measured, five classes with class constants (us per step, 4 blocks
// -> 5 blocks -> 6 blocks with the aliased observation tile): K=4 1M envs
// 58.3 -> 56.8 -> 54.8, 917k 52.8 -> 50.9 -> 51.1, 786k 47.7 -> 46.6 ->
// 46.0, 655k 39.45 -> 39.3 -> 39.7, 524k 32.96 -> 33.23 (5); K=8 1M 79.7 ->
// 79.55 -> 76.4; K=1 1M 45.4 -> 45.9 (5). So 6 where K >= 4 and the 6-block
// grid's blocks walk at least 1.25 tiles each, else 4.
int jit_step_min_blocks(int K, int n_tiles, int num_sms) {
  return K >= 4 && 4 * (int64_t)n_tiles >= 5 * (int64_t)(6 * num_sms) ? 6 : 4;
}

// The class-specialised one-class propeller step kernel for class table k
// (nt thrusters; ms: the multi-step instantiation; pm 0: the class's physics
// as literals too, 1: per-env physics from the parameter planes, the
// actuator tables as literals; compiled for min_blocks resident blocks per
// SM) on the current device, or null if it cannot be had (err says why).
const void* jit_step_kernel(const ClassK& k, int nt, bool ms, int pm, int min_blocks, std::string* err) {
  return jit_kernel(STEP, k, nt, ms, pm, min_blocks, err);
}

// The class-specialised adjoint kernel for class table k (nt thrusters).
const void* jit_adjoint_kernel(const ClassK& k, int nt, std::string* err) {
  return jit_kernel(ADJOINT, k, nt, false, 0, 0, err);
}

// Launch of a class-specialised kernel (same arguments and launch shape as
// the kernel built with the library).
cudaError_t launch_step_jit(const void* kern, const StepArgs& a, const ClassK& kc, int nt, int pm, int grid, bool dependent,
                            bool shared_sm, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = step_kernel_smem_jit(nt, pm);
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  int na = 0;
  if (shared_sm) {
    attr[na].id = cudaLaunchAttributePreferredSharedMemoryCarveout;
    attr[na].val.sharedMemCarveout = (unsigned)cudaSharedmemCarveoutMaxShared;
    ++na;
  }
  if (MG_USE_PDL && dependent) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  StepArgs aa = a;
  ClassK kk = kc;
  void* args[] = {&aa, &kk};
  return cudaLaunchKernelExC(&cfg, kern, args);
}

}  // namespace mg
