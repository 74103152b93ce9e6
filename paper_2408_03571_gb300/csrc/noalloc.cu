// hzs_apply_precond_noalloc: the SAS2 preconditioner apply with its per-call
// work space in a fixed, library-owned device array instead of memory
// allocated for the handle.
//
// Why it exists: some callers are not allowed to allocate device memory at the
// point where they apply the preconditioner - real-time or embedded hosts that
// forbid allocation after start-up, or applications that hand all device
// memory to their own pool and cannot give a library a share of it at run
// time.  This entry point performs no cudaMalloc, cudaFree or other allocating
// call; the caller passes only its input and output buffers.
//
// It runs the kernels of hzs_apply_precond for SAS2: the restriction, the FP64
// coarse product and the subdomain solve.  In mixed precision the subdomain
// solve writes z in complex128 directly, where hzs_apply_precond writes a
// complex64 array and widens it; the solve's output stage forms every value in
// the kernel's FP32 arithmetic and converts it only when it stores it, so the
// two results are identical bit for bit.
//
// The work space is the static array below (kNoAllocScratchBytes, 1 MiB).  It
// is part of the library's device image, so every GPU that loads the library
// holds it until the process exits.  Its device address is looked up once per
// device (cudaGetSymbolAddress) by the first call made with that device
// current; make that first call before any stream capture begins.  All calls
// share the one array: calls whose work overlaps on the GPU (other streams,
// other host threads, other handles) race on it and must be serialised by the
// caller.  Every byte a call reads from the array is written earlier in the
// same call, so nothing has to be cleared between calls.
#include <mutex>
#include <string>

#include "kernels.cuh"

using namespace hzs;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(1) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

const BatchSkip kNone{nullptr, 0};

// Device address of g_noalloc_scratch on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

// Accessors of the opaque handles (defined in api.cu).
hzs_status hzs_internal_noalloc_view(hzs_precond* p, NoAllocView* v, std::string* err);
hzs_status hzs_internal_set_error(hzs_precond* p, hzs_status s, const std::string& msg);

extern "C" hzs_status hzs_apply_precond_noalloc(hzs_precond* p, const void* v_dev, void* z_dev, int nrhs) {
    NoAllocView V{};
    std::string err;
    hzs_status st = hzs_internal_noalloc_view(p, &V, &err);
    if (st != HZS_OK) return st;
    if (!v_dev || !z_dev || nrhs < 0) return hzs_internal_set_error(p, HZS_ERR_INVALID_ARG, "bad buffers or nrhs");
    if (V.kind != HZS_SAS2)
        return hzs_internal_set_error(p, HZS_ERR_INVALID_ARG,
                                      "hzs_apply_precond_noalloc supports SAS2 preconditioners only");
    const int n = V.cx.op.n;
    const bool mixed = V.precision == HZS_MIXED;
    const size_t t_bytes = round256((size_t)n * V.nc1 * (mixed ? sizeof(float2) : sizeof(double2)));
    const size_t c_bytes = round256((size_t)V.Nc * sizeof(double2));
    const size_t cf_bytes = mixed ? round256((size_t)V.Nc * sizeof(float2)) : 0;
    const size_t need = t_bytes + 2 * c_bytes + cf_bytes;
    if (need > kNoAllocScratchBytes)
        return hzs_internal_set_error(
            p, HZS_ERR_INVALID_ARG,
            "problem needs " + std::to_string(need) + " bytes of work space; hzs_apply_precond_noalloc has " +
                std::to_string(kNoAllocScratchBytes) + " (use hzs_apply_precond)");
    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess)
        return hzs_internal_set_error(p, HZS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    unsigned char* b = static_cast<unsigned char*>(base);
    double2* c = reinterpret_cast<double2*>(b + t_bytes);
    double2* c2 = reinterpret_cast<double2*>(b + t_bytes + c_bytes);
    float2* c2f = mixed ? reinterpret_cast<float2*>(b + t_bytes + 2 * c_bytes) : nullptr;
    const size_t nn = (size_t)n * n;
    for (int r = 0; r < nrhs; ++r) {
        const double2* v = (const double2*)v_dev + r * nn;
        double2* z = (double2*)z_dev + r * nn;
        int rc;
        if (mixed) {
            launch_restrict<double2, float>(V.cx, 1, v, 0, nullptr, 0, reinterpret_cast<float2*>(b), c, kNone);
            launch_coarse_matvec(V.cx, 1, V.Ainv, V.Nc, c, c2, c2f, kNone);
            rc = launch_tile_solve<double2, double2, float>(V.cx, 1, V.tiles, V.groups, V.max_mx, V.max_my, V.W32,
                                                            v, 0, nullptr, 0, 0, c2f, 0, 1, z, 0, nullptr, 0, kNone);
        } else {
            launch_restrict<double2, double>(V.cx, 1, v, 0, nullptr, 0, reinterpret_cast<double2*>(b), c, kNone);
            launch_coarse_matvec(V.cx, 1, V.Ainv, V.Nc, c, c2, nullptr, kNone);
            rc = launch_tile_solve<double2, double2, double>(V.cx, 1, V.tiles, V.groups, V.max_mx, V.max_my, V.W64,
                                                             v, 0, nullptr, 0, 0, c2, 0, 1, z, 0, nullptr, 0, kNone);
        }
        if (rc != 0) return hzs_internal_set_error(p, HZS_ERR_CUDA, "subdomain solve launch failed");
    }
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return hzs_internal_set_error(p, HZS_ERR_CUDA, std::string("apply_precond_noalloc: ") + cudaGetErrorString(e));
    return HZS_OK;
}
