// odx_render_static: odx_render for callers that must not allocate device memory.
//
// Such callers cannot call odx_create either (it allocates the context's scratch).  This
// entry point keeps that scratch -- the ray-queue counter, the device statistics and the
// scene table -- in one file-scope device array that exists on every GPU which loads the
// library, from load until process exit, and it calls no cudaMalloc, cudaFree or other
// allocating routine.  Outputs and scene descriptions still come from the caller.
//
// In host code the array's name only stands for the symbol, not for its device address:
// the address is looked up once per device with cudaGetSymbolAddress (with that device
// current) and passed to the kernel as ordinary pointers.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "odx_internal.h"

namespace odx {
int32_t validate_scene_table(const odx_scene *scenes, int32_t n_scenes);
int32_t transfer_slots(int32_t emitter, int32_t n_freq);
}  // namespace odx

namespace {

using odx::DevScene;
using odx::DevStats;

// Layout of the static scratch: queue counter at 0, statistics at 64, scene table at 256.
constexpr size_t kQueueOffset = 0;
constexpr size_t kStatsOffset = 64;
constexpr size_t kScenesOffset = 256;
constexpr size_t kStaticBytes = 45056;
static_assert(kScenesOffset + ODX_STATIC_MAX_SCENES * sizeof(DevScene) <= kStaticBytes,
              "scene table does not fit the static scratch");
static_assert(sizeof(DevStats) <= kScenesOffset - kStatsOffset, "stats do not fit");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
struct DeviceSetup {
    bool ready;
    unsigned char *scratch;  // device address of g_static_scratch on this device
    int32_t num_sms;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Once per device, with that device current: find the array's device address.
int32_t device_setup(int dev, DeviceSetup *out)
{
    if (dev < 0 || dev >= kMaxDevices) return ODX_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &s = g_setup[dev];
    if (!s.ready) {
        int major = 0, minor = 0, sms = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return ODX_ERR_CUDA;
        if (major != 10 || minor != 3) return ODX_ERR_NO_DEVICE;
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || ptr == nullptr ||
            odx::prepare_fp64_kernels() != cudaSuccess)
            return ODX_ERR_CUDA;
        s.scratch = static_cast<unsigned char *>(ptr);
        s.num_sms = sms;
        s.ready = true;
    }
    *out = s;
    return ODX_OK;
}

}  // namespace

extern "C" int32_t odx_render_static(const odx_scene *scenes, int32_t n_scenes,
                                     odx_ray_record *records, double *image, void *stream)
{
    if (!scenes || n_scenes < 1 || !records) return ODX_ERR_INVALID_ARG;
    if (n_scenes > ODX_STATIC_MAX_SCENES) return ODX_ERR_TOO_LARGE;
    if (((uintptr_t)records & 15u) != 0 || (image && ((uintptr_t)image & 7u) != 0))
        return ODX_ERR_INVALID_ARG;
    const int32_t rc = odx::validate_scene_table(scenes, n_scenes);
    if (rc != ODX_OK) return rc;

    // scene table built on the host stack (no heap, no device allocation)
    DevScene table[ODX_STATIC_MAX_SCENES];
    const int64_t nf = odx::scene_planes(scenes[0]);
    int64_t ray = 0, img = 0;
    for (int k = 0; k < n_scenes; ++k) {
        const int64_t nk = (int64_t)scenes[k].n_alpha * scenes[k].n_beta;
        odx::fill_dev_scene(table[k], scenes[k], ray, nk, img);
        ray += nk;
        img += nf * nk;
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ODX_ERR_CUDA;
    DeviceSetup setup{};
    const int32_t src = device_setup(dev, &setup);
    if (src != ODX_OK) return src;

    cudaStream_t st = (cudaStream_t)stream;
    // the scene table below is copied from this call's stack frame: a graph captured from
    // the call would replay a copy from memory that no longer holds it
    cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &capture) != cudaSuccess) return ODX_ERR_CUDA;
    if (capture != cudaStreamCaptureStatusNone) return ODX_ERR_UNSUPPORTED;
    unsigned char *base = setup.scratch;
    // pageable source: the copy has taken the table before cudaMemcpyAsync returns
    if (cudaMemcpyAsync(base + kScenesOffset, table, n_scenes * sizeof(DevScene),
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(base, 0, kScenesOffset, st) != cudaSuccess)  // queue + statistics
        return ODX_ERR_CUDA;

    odx::TraceArgs a{};
    a.scenes = reinterpret_cast<const DevScene *>(base + kScenesOffset);
    a.n_scenes = n_scenes;
    a.list_mode = 0;
    a.rays = nullptr;
    a.n_total = ray;
    a.records = records;
    a.image = image;
    a.queue = reinterpret_cast<unsigned long long *>(base + kQueueOffset);
    a.stats = reinterpret_cast<DevStats *>(base + kStatsOffset);
    const odx_launch launch{128, 3, 0, 2, 16};
    a.chunk = launch.chunk;
    a.persistent = launch.persistent;
    a.fp64_batch = launch.fp64_batch;
    odx::set_launch_medium(a, table[0], odx::shared_medium(table, n_scenes));
    const int32_t slots = odx::transfer_slots(scenes[0].emitter, scenes[0].n_freq);
    const cudaError_t e =
        scenes[0].precision == ODX_MIXED
            ? odx::launch_trace_mixed(a, slots, launch, setup.num_sms, st)
            : odx::launch_trace_fp64(a, slots, launch, setup.num_sms, st);
    if (e == cudaErrorNotSupported) return ODX_ERR_UNSUPPORTED;
    return e == cudaSuccess ? ODX_OK : ODX_ERR_CUDA;
}
