// rgf_noalloc.cu -- rgf_conductance_noalloc: the conductance of one ribbon at
// several energies, with every scratch buffer taken from a fixed, statically
// sized device array instead of cudaMalloc.
//
// Who needs it: callers that may not allocate device memory themselves, for
// example a host application that has already reserved the device memory for
// its own pool and forbids further cudaMalloc, a plugin whose host hands it
// only pre-allocated buffers, or a loop that must not trigger the implicit
// device synchronisation that cudaMalloc / cudaFree can cause.  They pass
// their inputs and outputs as device pointers; everything else lives in the
// array below.
//
// The array (kScratchBytes, 64 MiB) is part of the library's device code: every
// GPU that loads that code holds it until the process exits.  CUDA loads device
// code lazily by default, so the array comes into being at this entry point's
// first call on a device (inside its cudaGetSymbolAddress), or when the context
// is created if CUDA_MODULE_LOADING=EAGER is set; a caller that reserves the
// device memory for its own pool should make one call before doing so.  The
// first call on a device looks the address up and caches it (make that call
// before any stream capture); after cudaDeviceReset of that device the cached
// address is stale, so the entry point must not be used again in that process.
// All calls share the array, and it keeps the previous call's contents; calls
// whose work overlaps on the GPU (concurrent streams, or a second call before
// the first has finished on another stream) race on it.  Each call writes its
// own descriptors into the array with a kernel (nothing is copied from host
// memory) and every part of the array it reads is written earlier in the same
// call.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "rgf.h"
#include "rgf_internal.h"

namespace rgf {
void set_last_error(const std::string& msg);
}

namespace {

constexpr size_t kScratchBytes = 64ull << 20;   // 64 MiB
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

rgf_status nfail(rgf_status st, const std::string& msg) {
    rgf::set_last_error("rgf_conductance_noalloc: " + msg);
    return st;
}

// Device address of g_scratch on the current device; set up once per device.
cudaError_t scratch_address(int dev, void** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// Chain and lead descriptors of call i (one per energy) written on the device
// from the call's arguments, so that a call copies nothing from the host.  A
// non-finite energy is reported by the lead kernel as RGF_EINVAL.
__global__ void noalloc_setup(rgf::ChainDev* chains, rgf::LeadDev* leads, int* order,
                              int* lead_status, const double* onsite, const uint8_t* removed,
                              int N, int L, double t, const double* E, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        rgf::ChainDev& ch = chains[i];
        ch.eps = onsite;
        ch.rem = removed;
        ch.N = N;
        ch.L = L;
        ch.t = t;
        ch.E = E[i];
        ch.lead = i;
        ch.ws_off = (size_t)i * rgf::sweep_ws_elems(N);
        ch.grad_off = 0;
        rgf::default_sched(ch);
        rgf::LeadDev& ld = leads[i];
        ld.N = N;
        ld.t = t;
        ld.E = E[i];
        ld.off = (size_t)i * rgf::lead_out_elems(N);
        ld.ws_off = (size_t)i * rgf::lead_ws_elems(N);
        order[i] = i;
        lead_status[2 * i] = lead_status[2 * i + 1] = 0;
    }
}

}  // namespace

extern "C" rgf_status rgf_conductance_noalloc(int N, int L, double t, const double* onsite_dev,
                                              const uint8_t* removed_dev, const double* E_dev,
                                              int nE, double eta_device, double eta_lead,
                                              int precision, void* stream, double* T_dev,
                                              int32_t* status_dev) {
    if (nE < 0) return nfail(RGF_EINVAL, "nE < 0");
    if (nE == 0) return RGF_OK;
    if (N < 2 || N > 2047 || L < 1 || !std::isfinite(t) || t == 0.0)
        return nfail(RGF_EINVAL, "bad N, L or t");
    if (!onsite_dev || !E_dev || !T_dev) return nfail(RGF_EINVAL, "NULL device pointer");
    if (precision != RGF_FP64 && precision != RGF_MIXED && precision != RGF_MIXED_TC &&
        precision != RGF_FP64_TC)
        return nfail(RGF_EINVAL, "unknown precision");
    if (!(eta_device >= 0.0) || !(eta_lead > 0.0) || !std::isfinite(eta_device) ||
        !std::isfinite(eta_lead))
        return nfail(RGF_EINVAL, "eta_device must be >= 0 and eta_lead > 0 (finite)");

    // Scratch layout (each part 256-byte aligned): descriptors | lead status |
    // lead workspace | lead output | sweep workspace.
    const size_t n = (size_t)nE;
    const size_t b_chain = n * sizeof(rgf::ChainDev), b_lead = n * sizeof(rgf::LeadDev);
    const size_t b_order = n * sizeof(int);
    const size_t o_chain = 0, o_lead = up256(o_chain + b_chain), o_order = up256(o_lead + b_lead);
    const size_t o_lst = up256(o_order + b_order);
    const size_t o_lws = up256(o_lst + 2 * n * sizeof(int));
    const size_t o_lout = up256(o_lws + n * rgf::lead_ws_elems(N) * 16);
    const size_t o_ws = up256(o_lout + n * rgf::lead_out_elems(N) * 16);
    const size_t total = o_ws + n * rgf::sweep_ws_elems(N) * 16;
    if (total > kScratchBytes)
        return nfail(RGF_EINVAL, "needs " + std::to_string(total) + " bytes of scratch for N = " +
                                     std::to_string(N) + ", " + std::to_string(nE) +
                                     " energies; the fixed limit is " +
                                     std::to_string(kScratchBytes) + " bytes (64 MiB): use fewer "
                                     "energies per call or rgf_conductance_dev");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return nfail(RGF_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return nfail(RGF_EINVAL, "device ordinal out of range");
    void* base = nullptr;
    e = scratch_address(dev, &base);
    if (e != cudaSuccess)
        return nfail(RGF_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    unsigned char* sp = static_cast<unsigned char*>(base);

    cudaStream_t st = (cudaStream_t)stream;
    auto* dchains = reinterpret_cast<rgf::ChainDev*>(sp + o_chain);
    auto* dleads = reinterpret_cast<rgf::LeadDev*>(sp + o_lead);
    auto* dorder = reinterpret_cast<int*>(sp + o_order);
    auto* dlst = reinterpret_cast<int*>(sp + o_lst);
    noalloc_setup<<<(nE + 255) / 256, 256, 0, st>>>(dchains, dleads, dorder, dlst, onsite_dev,
                                                     removed_dev, N, L, t, E_dev, nE);
    e = cudaGetLastError();
    if (e != cudaSuccess) return nfail(RGF_ECUDA, cudaGetErrorString(e));
    const int Kmax = rgf::col_KL(N);
    // as rgf_conductance_dev: the tensor-core layout of the widest columns
    // exceeds a block's shared memory, and their products run on the pipes
    if ((precision == RGF_MIXED_TC || precision == RGF_FP64_TC) && !rgf::tc_layout_fits(Kmax))
        precision = precision == RGF_MIXED_TC ? RGF_MIXED : RGF_FP64;
    e = rgf::launch_lead(dleads, nE, Kmax, eta_lead, sp + o_lws, sp + o_lout, dlst, nullptr, st);
    if (e != cudaSuccess) return nfail(RGF_ECUDA, cudaGetErrorString(e));
    e = rgf::launch_prep(precision, dchains, dorder, nE, Kmax, eta_device, sp + o_lout, dlst, dleads,
                         sp + o_ws, st);
    if (e == cudaSuccess)
        e = rgf::launch_half(precision, dchains, dorder, nE, Kmax, eta_device, sp + o_lout, dlst,
                             dleads, sp + o_ws, st);
    if (e == cudaSuccess)
        e = rgf::launch_merge(precision, dchains, dorder, nE, Kmax, eta_device, sp + o_lout, dlst,
                              dleads, sp + o_ws, T_dev, status_dev, st);
    if (e != cudaSuccess) return nfail(RGF_ECUDA, cudaGetErrorString(e));
    return RGF_OK;
}
