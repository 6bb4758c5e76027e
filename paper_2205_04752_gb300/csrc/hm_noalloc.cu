// hm_noalloc.cu -- an H-matrix-vector product that allocates nothing.
//
// Some callers cannot allocate device memory at the time they need a
// product: code that runs under a fixed, pre-reserved memory budget (a
// real-time or embedded host loop, a plug-in inside another framework's
// allocator), or code paths where calling cudaMalloc would synchronise the
// device or is simply not permitted.  hm_matvec itself allocates nothing per
// call, but it uses the workspace that hm_aca_assemble reserved inside the
// matrix; hm_matvec_noalloc instead takes its workspace from one file-scope
// device array of fixed size that is part of the loaded library.
//
// The array is module memory: every GPU on which the library's device code
// is loaded holds kNoAllocScratchBytes of it until the process exits.  All
// calls share it: two calls whose kernels overlap on the device (different
// streams, different host threads, or different matrices) race on it and
// give wrong results.  Nothing in it has to start at zero: every call
// overwrites each scratch element before reading it.
#include <algorithm>

#include "hm_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the array on the current device.  In host code the name
// g_noalloc_scratch is only a host-side stand-in for the symbol, never a
// device address, so the address is looked up with the calling device
// current.  It is looked up on every call (cheap once the module is loaded):
// a cached address would go stale if the caller reset the device, which
// unloads the module and may place the array elsewhere on reload.  The first
// call on a device may load the library's device code there.
int scratch_address(void** out)
{
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return hm::cuda_check(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                              "cudaGetSymbolAddress(g_noalloc_scratch)");
    *out = p;
    return HM_OK;
}

}  // namespace

extern "C" int hm_matvec_noalloc(const hm_matrix* H, const double* x, double* y, int32_t nrhs,
                                 int64_t ld, int32_t form, void* stream)
{
    using namespace hm;
    if (!H || !x || !y) return fail(HM_EINVAL, "hm_matvec_noalloc: NULL argument");
    if (H->rect) return fail(HM_EINVAL, "hm_matvec_noalloc: an evaluation operator (hm_build_point_tree) has only hm_eval_points and hm_amvm");
    if (nrhs < 1 || nrhs > H->max_rhs)
        return fail(HM_EINVAL, "hm_matvec_noalloc: nrhs=%d outside 1..%d", nrhs, H->max_rhs);
    if (ld < 3 * H->M)
        return fail(HM_EINVAL, "hm_matvec_noalloc: ld=%lld < 3M=%lld", (long long)ld,
                    (long long)(3 * H->M));
    if (form < HM_FP64 || form >= HM_NFORMS) return fail(HM_EINVAL, "hm_matvec_noalloc: unknown form %d", form);
    if (!H->packed[form])
        return fail(HM_EINVAL, "hm_matvec_noalloc: form %d not packed (call hm_pack)", form);
    const char* xb = (const char*)x;
    const char* yb = (const char*)y;
    size_t span = ((size_t)(nrhs - 1) * ld + 3 * H->M) * sizeof(double);
    if (xb < yb + span && yb < xb + span) return fail(HM_EINVAL, "hm_matvec_noalloc: x and y overlap");
    const size_t need = matvec_scratch_bytes(*H, nrhs, form);
    if (need > kNoAllocScratchBytes)
        return fail(HM_EINVAL,
                    "hm_matvec_noalloc: this product needs %zu bytes of scratch but the static "
                    "scratch holds %zu; use hm_matvec or fewer right-hand sides",
                    need, kNoAllocScratchBytes);
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    const Scratch scr = make_scratch(*H, nrhs, form, base);
    return matvec_device_scratch(*H, x, y, nrhs, ld, form, (cudaStream_t)stream, scr);
}
