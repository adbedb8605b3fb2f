// ncpadj_elastic_solve_noalloc: y = A^{-1} x without allocating device memory during the call.
//
// Some callers cannot let a library allocate device memory once they are running: programs
// whose device memory is reserved up front by their own pool or allocator, and loops with hard
// latency limits where a cudaMalloc (which may synchronise the device and take milliseconds) is
// not acceptable.  For them this entry point keeps its two intermediate vectors -- x permuted to
// elimination order, and S P x of the sparse-inverse product A^{-1} = P^T S^T S P -- in a static
// device array instead of the scene's grow-on-demand workspace.  The caller still provides x and
// y; the scene's arrays were allocated when the scene was created.
//
// The array lives in this file's own module.  CUDA loads a module's device memory lazily, when one
// of its symbols is first used, so ncpadj_ctx_create looks the array up (noalloc_prepare): the
// array is then allocated while the context is created, and the solve itself allocates nothing.
#include <mutex>

#include "internal.h"
#include "kernels.cuh"

namespace ncpadj {
namespace {

// Largest scene (in vertices) this entry point accepts: the scratch holds two [n_verts][3]
// float64 vectors, 12 MiB.  Every GPU on which a context is created holds the array until the
// process exits.
constexpr int kNoAllocMaxVerts = 262144;
__device__ __align__(256) double g_noalloc_scratch[2 * 3 * (size_t)kNoAllocMaxVerts];  // w, then x permuted

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

// In host code the array's name is only a host-side stand-in; the kernels need its device
// address, looked up once per device with that device current.
double* scratch_address(int device) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    NCPADJ_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_addr[device] = static_cast<double*>(p);
  }
  return g_scratch_addr[device];
}

}  // namespace

void noalloc_prepare(int device) {
  NCPADJ_REQUIRE(device >= 0 && device < kMaxDevices, "device ordinal out of range");
  scratch_address(device);
}

}  // namespace ncpadj

using namespace ncpadj;

extern "C" ncpadj_status ncpadj_elastic_solve_noalloc(ncpadj_ctx ctx, ncpadj_scene scene, const double* x, double* y,
                                                      void* stream) {
  set_error("");
  try {
    NCPADJ_REQUIRE(ctx && scene && x && y && x != y, "NULL or aliased argument");
    NCPADJ_REQUIRE(ctx->c.device >= 0 && ctx->c.device < kMaxDevices, "device ordinal out of range");
    Scene& S = scene->s;
    NCPADJ_REQUIRE(S.nv <= kNoAllocMaxVerts,
                   "scene has " + std::to_string(S.nv) + " vertices; ncpadj_elastic_solve_noalloc supports at most " +
                       std::to_string(kNoAllocMaxVerts));
    NCPADJ_CUDA_TRY(cudaSetDevice(ctx->c.device));
    double* w = scratch_address(ctx->c.device);  // looked up by ncpadj_ctx_create: no allocation here
    SinvArgs a{S.nv, S.S_ptr.as<int64_t>(), S.S_c0.as<int32_t>(), S.S_val.as<double>(), S.St_ptr.as<int64_t>(),
               S.St_col.as<int32_t>(), S.St_val.as<double>(), S.perm.as<int32_t>(), S.nS_chunks, S.nSt_chunks,
               S.S_crow.as<int32_t>(), S.St_crow.as<int32_t>(), S.S_cbeg.as<int64_t>(), S.S_cend.as<int64_t>(),
               S.St_cbeg.as<int64_t>(), S.St_cend.as<int64_t>()};
    a.chunk = S.chunk;
    a.xpos = w + 3 * (size_t)kNoAllocMaxVerts;
    // the product zeroes the scratch before accumulating into it, so earlier calls leave nothing behind
    launch_ainv(a, x, w, y, (cudaStream_t)stream);
    NCPADJ_CUDA_TRY(cudaGetLastError());
    return NCPADJ_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.status;
  } catch (const std::exception& e) {
    set_error(e.what());
    return NCPADJ_ERR_INVALID_ARG;
  }
}
