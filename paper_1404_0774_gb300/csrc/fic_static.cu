// fic_encode_static: the encode pipeline with its scratch memory in a fixed
// device array that lives inside this library, for callers that may not
// allocate device memory themselves.
//
// Who needs this: code that runs where asking the CUDA allocator for memory
// is not allowed or not acceptable -- a plug-in whose host application owns
// and budgets all device memory, a real-time pipeline that reserves every
// buffer at start-up so that no allocation can stall a frame later, or a
// process running under a hard device-memory cap set by someone else.  Such a
// caller can neither pass a workspace it allocated nor let fic_encode
// allocate one.  This entry point uses instead a static array of
// FIC_STATIC_SCRATCH_BYTES (32 MiB) that every GPU which loads the library
// holds until the process exits.
#include <cuda.h>

#include <mutex>

#include "fic_internal.cuh"

namespace {

constexpr size_t kStaticBytes = FIC_STATIC_SCRATCH_BYTES;

// The scratch.  In host code this name is only a host-side stand-in for the
// device array, never a device address: the address a kernel may use comes
// from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Per device: the array's device address and the unique id of the context it
// was looked up in.  A context that is destroyed and created again (e.g.
// after cudaDeviceReset) has a new id, so the stale address is dropped.
struct Entry {
    void *addr;
    unsigned long long ctx_id;
};
Entry g_entry[kMaxDevices] = {};

typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context, or 0 if none is
// current or the driver does not report one.
unsigned long long current_ctx_id()
{
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qb == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<PfnCtxGetCurrent>(a);
            get_id = reinterpret_cast<PfnCtxGetId>(b);
        }
        cudaGetLastError();
    }
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of g_scratch on the current device.  Looked up (with that
// device current) on the first call for the device and again whenever its
// context has changed since; a failed lookup leaves no cached entry.  Returns
// nullptr on failure.
void *scratch_address()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    Entry &e = g_entry[dev];
    const unsigned long long id = current_ctx_id();
    if (e.addr && id != 0 && id == e.ctx_id) return e.addr;
    e = Entry{nullptr, 0};
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return nullptr;
    }
    // the lookup made the device's context current if none was; without a
    // context id the address is not cached (looked up on every call)
    const unsigned long long id2 = current_ctx_id();
    if (id2 != 0) e = Entry{ptr, id2};
    return ptr;
}

}  // namespace

extern "C" {

int fic_encode_static(const void *img, int w, int h, int pitch_px, const fic_params *p, fic_map *maps,
                      int maps_cap, int *n_maps, void *stream)
{
    if (!img || !maps || !p) return FIC_ERR_BAD_ARG;
    if (p->flags & FIC_FLAG_PHASE_TIMING) return FIC_ERR_BAD_ARG;  // timing events would be created
    size_t need = 0;
    const int rc = fic_encode_workspace_size(w, h, p, &need);  // host-only size check, no device call
    if (rc != FIC_OK) return rc;
    if (need > kStaticBytes) return FIC_ERR_CAPACITY;
    void *ws = scratch_address();
    if (!ws) return FIC_ERR_CUDA;
    return fic::encode_with_workspace(img, w, h, pitch_px, p, maps, maps_cap, n_maps, ws, kStaticBytes, stream);
}

}  // extern "C"
