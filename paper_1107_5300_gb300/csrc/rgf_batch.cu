// rgf_batch.cu -- the persistent schedule of the forward sweep: one kernel
// whose blocks take the halves of the chains from a device work queue (the
// method and the device bodies are in rgf_half.cuh).
#include "rgf_half.cuh"

namespace rgf {

// Persistent schedule: gridDim.x blocks (at most one per SM) take halves from
// the work queue (queue[0] = next item; item 2i + h = half h of chain
// order[i], so the halves go out longest chain first) until it is empty.  A
// block prepares its half's end column, runs its recursion, and counts the
// half done on its chain (queue[1 + ci]); the block that brings the count to
// two -- its partner half is complete by then -- joins the halves and writes T
// and the status word.  Nothing waits: a block never spins on another block,
// the queue and the counters only hand out work.  The release of a finished
// half (its workspace, by every thread) to the joining block is the block
// barrier, a device-scope fence and the counter's atomic on one side, the
// atomic and a fence on the other.  With TC the block holds TMEM for the
// whole launch.
template <class R, bool TC>
__global__ void __launch_bounds__(NT, 1) batch_kernel(SweepArgs a, int bm, int* queue) {
    __shared__ int s_item, s_join;
    tc::State tst;
    if constexpr (TC) {
        SweepSmem<R> s = carve<R>(rgf_dyn_smem, a.Kmax, TC, bm);
        tc_attach<R>(a.Kmax, s, tst);
    }
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&queue[0], 1);
        __syncthreads();
        const int item = s_item;
        if (item >= 2 * a.nchains) break;
        {
            const int ci = a.order[item >> 1], h = item & 1;
            if (lead_state(a.lead_status, a.chains[ci].lead) == ST_OK) {
                prep_body<R>(a, ci, h, bm);
                half_body<R, TC>(a, ci, h, bm, &tst);
            }
        }
        // the chain is looked up again from the item in shared memory, so that
        // nothing of the loop stays live in registers across the half sweep
        if (threadIdx.x == 0) {
            const int cj = a.order[*(volatile int*)&s_item >> 1];
            __threadfence();
            s_join = cj | (atomicAdd(&queue[1 + cj], 1) << 30);
            __threadfence();
        }
        __syncthreads();
        {
            const int j = *(volatile int*)&s_join;
            if ((j >> 30) == 1) merge_body<R>(a, j & ((1 << 30) - 1), bm);
        }
        __syncthreads();                 // s_item and s_join are rewritten next
    }
    if constexpr (TC) tc::teardown(tst.ar);
}

cudaError_t configure_batch(int precision, int Kmax) {
    const size_t f64 = f64_smem(precision, Kmax), rec = rec_smem(precision, Kmax);
    const size_t both = rec > f64 ? rec : f64;
    auto kern = precision == 0   ? batch_kernel<double, false>
                : precision == 3 ? batch_kernel<double, true>
                : precision == 2 ? batch_kernel<df32, true>
                                 : batch_kernel<df32, false>;
    return set_smem(kern, both);
}

cudaError_t launch_batch(int precision, const ChainDev* chains, const int* order, int nchains,
                         int Kmax, double eta_device, const void* leadout, const int* lead_status,
                         const LeadDev* leads, void* ws, double* T, int32_t* status, int* queue,
                         int nsm, cudaStream_t st) {
    if (nchains <= 0) return cudaSuccess;
    cudaError_t e = configure_batch(precision, Kmax);
    if (e != cudaSuccess) return e;
    const SweepArgs a = make_args(chains, order, nchains, Kmax, eta_device, leadout, lead_status,
                                  leads, ws, T, status);
    const size_t f64 = f64_smem(precision, Kmax), rec = rec_smem(precision, Kmax);
    const int grid = nsm < 2 * nchains ? (nsm > 0 ? nsm : 1) : 2 * nchains;
    auto kern = precision == 0   ? batch_kernel<double, false>
                : precision == 3 ? batch_kernel<double, true>
                : precision == 2 ? batch_kernel<df32, true>
                                 : batch_kernel<df32, false>;
    kern<<<grid, NT, rec > f64 ? rec : f64, st>>>(a, launch_panel(precision, Kmax), queue);
    return cudaGetLastError();
}

}  // namespace rgf
