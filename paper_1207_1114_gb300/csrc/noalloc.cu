// noalloc.cu -- fastpfp_project_noalloc: the successive projection of
// fastpfp_project for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: a plugin that a host
// application hands a fixed device-memory arena (the application accounts
// for every byte on the GPU and refuses allocations made behind its back),
// or a real-time loop that forbids allocation after start-up (cudaMalloc can
// block and synchronise the device for an unbounded time).  They cannot
// create a handle (fastpfp_create allocates), so this entry point needs
// none.  The caller passes the matrix Y in and gets it
// back in place; the only scratch the projection kernel needs beyond Y (its
// rotating column-sum accumulators, the FP64 totals, the round maxima and
// the barrier/control words) lives in one file-scope device array of fixed
// size, present on every GPU that loads this library until the process
// exits.  The kernel is the same one fastpfp_project launches.
#include <cstddef>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "internal.h"

using namespace fpfp;

namespace {

constexpr int kNoallocMaxN = 4096;   // largest N this entry point accepts
constexpr int kMaxDevices = 64;
constexpr size_t kCtrlBytes = (sizeof(Ctrl) + 255) & ~size_t(255);
constexpr size_t kColBytes = (size_t)kNoallocMaxN * (3 * sizeof(float) + sizeof(double));   // colbuf_bytes
constexpr size_t kScratchBytes = kCtrlBytes + kColBytes + 256 + 256;

// The shared scratch.  Host code must not use this name as a device address:
// on the host it is only a stand-in, and the device address is obtained with
// cudaGetSymbolAddress (below) once per device.
static __device__ __align__(256) unsigned char fastpfp_noalloc_scratch[kScratchBytes];

struct DeviceSetup {
    bool ready = false;
    unsigned char* scratch = nullptr;  // device address of fastpfp_noalloc_scratch
    int num_sms = 0;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Once per device, with that device current: resolve the scratch address,
// read the SM count and set the kernel's shared-memory limit.
int setup_device(int dev, DeviceSetup** out) {
    if (dev < 0 || dev >= kMaxDevices) return FASTPFP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup& d = g_setup[dev];
    if (!d.ready) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, fastpfp_noalloc_scratch) != cudaSuccess || !p)
            return FASTPFP_ERR_CUDA;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return FASTPFP_ERR_CUDA;
        if (pd_configure() != cudaSuccess) return FASTPFP_ERR_CUDA;
        d.scratch = static_cast<unsigned char*>(p);
        d.num_sms = sms;
        d.ready = true;
    }
    *out = &d;
    return FASTPFP_OK;
}

}  // namespace

extern "C" int fastpfp_project_noalloc(void* stream, float* Y, int N, double tol, int max_iter,
                                       int* iters, double* last_delta) {
    if (!Y || N < 1 || max_iter < 1 || !(tol >= 0.0)) return FASTPFP_ERR_ARG;
    if (N > kNoallocMaxN) return FASTPFP_ERR_SIZE;
    if ((N & 3) != 0 || (reinterpret_cast<uintptr_t>(Y) & 15) != 0) return FASTPFP_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FASTPFP_ERR_CUDA;
    DeviceSetup* d = nullptr;
    int rc = setup_device(dev, &d);
    if (rc != FASTPFP_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;

    Ctrl* ctrl = reinterpret_cast<Ctrl*>(d->scratch);
    float* colbuf = reinterpret_cast<float*>(d->scratch + kCtrlBytes);
    double* sbuf = reinterpret_cast<double*>(d->scratch + kCtrlBytes + kColBytes);
    unsigned* dbuf = reinterpret_cast<unsigned*>(d->scratch + kCtrlBytes + kColBytes + 256);
    // the previous call's contents stay in the array: clear what must start at zero
    if (cudaMemsetAsync(ctrl, 0, offsetof(Ctrl, inner_trace), s) != cudaSuccess ||
        cudaMemsetAsync(colbuf, 0, colbuf_bytes(N), s) != cudaSuccess ||
        cudaMemsetAsync(sbuf, 0, 3 * sizeof(double), s) != cudaSuccess ||
        cudaMemsetAsync(dbuf, 0, kDbufWords * sizeof(unsigned), s) != cudaSuccess)
        return FASTPFP_ERR_CUDA;

    PdLaunch L;
    pd_plan(N, d->num_sms, &L);
    PdParams P{};
    P.Y = Y;
    P.N = N;
    P.ldy = L.ldy;  // == N since N is a multiple of 4
    P.m = N;
    P.tol_inner = tol;
    P.max_inner = max_iter;
    P.colbuf = colbuf;
    P.sbuf = sbuf;
    P.dbuf = dbuf;
    P.ctrl = ctrl;
    P.timeout_ns = 2000ll * 1000000ll;
    P.rpc = L.rpc;
    P.mode = kPdProjectOnly;
    if (pd_launch(L, P, s) != cudaSuccess) return FASTPFP_ERR_CUDA;

    struct { int error, last_inner; double last_delta; } out{};
    if (cudaMemcpyAsync(&out.error, &ctrl->error, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&out.last_inner, &ctrl->last_inner, sizeof(int), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(&out.last_delta, &ctrl->last_delta, sizeof(double), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return FASTPFP_ERR_CUDA;
    if (iters) *iters = out.last_inner;
    if (last_delta) *last_delta = out.last_delta;
    return out.error != 0 ? out.error : FASTPFP_OK;
}
