// Potentials given at run time.  PyCOOL turns the potential strings of a
// model file into CUDA kernels with SymPy and jinja2 templates, compiled by
// PyCUDA, and writes them out for inspection (Sec. 2.4).  Here the caller
// gives the potential and its derivatives as C expressions in the fields f0,
// f1 and the parameters p[0..7] (pycool_model_define); NVRTC compiles them
// into one elementwise kernel for the device the library runs on, which a
// stage launches between the library's own drift and kick kernels
// (sweep.cuh: rt_drift, rt_kick).  The generated source can be read back
// (pycool_model_source).
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pycool.h"
#include "runtime.h"
#include "sweep.cuh"

#define PYCOOL_API extern "C" __attribute__((visibility("default")))

namespace pycool {

namespace {

struct RtModel {
  int nf = 0;
  std::string source;
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kern = nullptr;
};

std::mutex g_rt_mu;
std::vector<RtModel> g_rt;   // entry i is model id kRuntimeModelBase + i

struct RtParams {
  double p[8];
};

std::string make_source(int nf, const char* V, const char* const* dV) {
  std::string s =
      "// generated by pycool_model_define: V and dV/dphi_i of a potential given at run time\n"
      "struct RtParams { double p[8]; };\n"
      "extern \"C\" __global__ void pycool_model_kernel(const double* __restrict__ phis,\n"
      "    double* __restrict__ dV, double* __restrict__ V, long long S, const RtParams prm) {\n"
      "  const double* p = prm.p;\n"
      "  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S;\n"
      "       i += (long long)gridDim.x * blockDim.x) {\n"
      "    const double f0 = phis[i];\n";
  if (nf == 2) s += "    const double f1 = phis[S + i];\n";
  s += "    V[i] = (" + std::string(V) + ");\n";
  s += "    dV[i] = (" + std::string(dV[0]) + ");\n";
  if (nf == 2) s += "    dV[S + i] = (" + std::string(dV[1]) + ");\n";
  s += "  }\n}\n";
  return s;
}

}  // namespace

int runtime_model_nfields(int id) {
  std::lock_guard<std::mutex> lk(g_rt_mu);
  const int i = id - kRuntimeModelBase;
  return (i >= 0 && i < (int)g_rt.size()) ? g_rt[i].nf : -1;
}

// The compiled potential of a runtime-model simulation at the fields `phis`
// (N_f n^3 float64 values): V' into d.rt_dV, V into d.rt_V.
cudaError_t launch_runtime_potential(const SimDesc& d, const double* phis, cudaStream_t s) {
  cudaKernel_t kern = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_rt_mu);
    if (d.rt_index < 0 || d.rt_index >= (int)g_rt.size()) return cudaErrorInvalidValue;
    kern = g_rt[d.rt_index].kern;
  }
  double* dV = d.rt_dV;
  double* V = d.rt_V;
  long long S = (long long)d.S;
  RtParams prm;
  for (int i = 0; i < 8; ++i) prm.p[i] = d.params[i];
  void* args[] = {(void*)&phis, (void*)&dV, (void*)&V, (void*)&S, (void*)&prm};
  return cudaLaunchKernel((const void*)kern, dim3(152 * 8), dim3(256), args, 0, s);
}

// One stage of a runtime-model simulation: drift, the compiled potential, kick.
cudaError_t launch_runtime_stage(const SimDesc& d, const LaunchTable& t, int grid,
                                 cudaStream_t s) {
  {
    std::lock_guard<std::mutex> lk(g_rt_mu);
    if (d.rt_index < 0 || d.rt_index >= (int)g_rt.size()) return cudaErrorInvalidValue;
  }
  if (grid == 0) return cudaSuccess;
  const unsigned eg = 152 * 8;
  if (d.model == M_RUNTIME1) rt_drift<M_RUNTIME1><<<eg, kThreads, 0, s>>>(t);
  else rt_drift<M_RUNTIME2><<<eg, kThreads, 0, s>>>(t);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_runtime_potential(d, d.rt_phis, s);
  if (e != cudaSuccess) return e;
#define PYCOOL_RT(M, ST)                                              \
  if (d.model == M && d.stencil == ST) {                              \
    rt_kick<M, ST><<<grid, kThreads, 0, s>>>(t);                      \
    return cudaGetLastError();                                        \
  }
  PYCOOL_RT(M_RUNTIME1, 7) PYCOOL_RT(M_RUNTIME1, 27) PYCOOL_RT(M_RUNTIME1, 13)
  PYCOOL_RT(M_RUNTIME2, 7) PYCOOL_RT(M_RUNTIME2, 27) PYCOOL_RT(M_RUNTIME2, 13)
#undef PYCOOL_RT
  return cudaErrorInvalidValue;
}

}  // namespace pycool

using namespace pycool;

PYCOOL_API pycool_status pycool_model_define(int32_t nf, const char* V, const char* const* dV,
                                             int32_t* model_id) {
  if (!model_id || (nf != 1 && nf != 2) || !V || !dV || !dV[0] || (nf == 2 && !dV[1]))
    return PYCOOL_E_INVALID;
  {
    std::lock_guard<std::mutex> lk(g_rt_mu);
    if ((int)g_rt.size() >= kRuntimeModelMax) return PYCOOL_E_NOMEM;
  }
  RtModel m;
  m.nf = nf;
  m.source = make_source(nf, V, dV);
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, m.source.c_str(), "pycool_model.cu", 0, nullptr, nullptr) !=
      NVRTC_SUCCESS)
    return PYCOOL_E_CUDA;
  const char* opts[] = {"--gpu-architecture=sm_103a", "--std=c++17"};
  const nvrtcResult cr = nvrtcCompileProgram(prog, 2, opts);
  if (cr != NVRTC_SUCCESS) {
    size_t n = 0;
    nvrtcGetProgramLogSize(prog, &n);
    std::string log(n, '\0');
    if (n) nvrtcGetProgramLog(prog, &log[0]);
    std::fprintf(stderr, "pycool_model_define: the expressions do not compile:\n%s\n",
                 log.c_str());
    nvrtcDestroyProgram(&prog);
    return PYCOOL_E_INVALID;
  }
  size_t cubin_size = 0;
  std::vector<char> cubin;
  if (nvrtcGetCUBINSize(prog, &cubin_size) != NVRTC_SUCCESS || cubin_size == 0) {
    nvrtcDestroyProgram(&prog);
    return PYCOOL_E_CUDA;
  }
  cubin.resize(cubin_size);
  const nvrtcResult gr = nvrtcGetCUBIN(prog, cubin.data());
  nvrtcDestroyProgram(&prog);
  if (gr != NVRTC_SUCCESS) return PYCOOL_E_CUDA;
  if (cudaLibraryLoadData(&m.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) !=
          cudaSuccess ||
      cudaLibraryGetKernel(&m.kern, m.lib, "pycool_model_kernel") != cudaSuccess) {
    cudaGetLastError();
    if (m.lib) cudaLibraryUnload(m.lib);
    return PYCOOL_E_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_rt_mu);
  g_rt.push_back(m);
  *model_id = kRuntimeModelBase + (int32_t)g_rt.size() - 1;
  return PYCOOL_OK;
}

PYCOOL_API pycool_status pycool_model_source(int32_t model_id, char* buf, size_t cap,
                                             size_t* len) {
  std::lock_guard<std::mutex> lk(g_rt_mu);
  const int i = model_id - kRuntimeModelBase;
  if (i < 0 || i >= (int)g_rt.size()) return PYCOOL_E_INVALID;
  const std::string& src = g_rt[i].source;
  if (len) *len = src.size();
  if (buf) {
    if (cap < src.size() + 1) return PYCOOL_E_INVALID;
    std::memcpy(buf, src.c_str(), src.size() + 1);
  }
  return PYCOOL_OK;
}
