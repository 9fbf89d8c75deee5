// rgf_internal.h -- descriptors shared by the host driver (rgf_api.cu) and the
// kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace rgf {

// Column slicing of a unit cell: the 2N orbitals of a cell split into four
// columns at x = 0, a, 1.5a, 2.5a (no hopping inside a column).  Element p of
// column c is orbital 4p + c; columns 0, 1 hold KL = ceil(N/2) orbitals
// (even rows), columns 2, 3 hold KR = floor(N/2) (odd rows).
__host__ __device__ inline int col_KL(int N) { return (N + 1) / 2; }
__host__ __device__ inline int col_KR(int N) { return N / 2; }

// One lead problem: pristine ribbon of N dimer lines at energy E.
struct LeadDev {
    int N;
    double t, E;
    size_t off;      // offset (in 16-byte complex elements) of this problem's output:
                     // Sigma_L [KL*KL], Sigma_R [KR*KR], Gamma_L [KL*KL], Gamma_R [KR*KR]
                     // (site basis of the lead-attached columns), then U_even [KL*KL],
                     // U_odd [KR*KR] (the transverse-mode vectors, real parts; row = atom,
                     // column = mode) and w [KL] (the mode self-energies tau_p^2 g_p), so
                     // that Sigma_L = U_even diag(w) U_even^T, Sigma_R = U_odd diag(w) U_odd^T
    size_t ws_off;   // offset (16-byte elements) of its decimation workspace
};

// One chain: a ribbon at one energy.
struct ChainDev {
    const double* eps;      // [L][2N] on-site energies (device)
    const uint8_t* rem;     // [L][2N] removal mask (device) or nullptr
    int N, L;
    double t, E;
    int lead;               // index of its lead problem
    size_t ws_off;          // offset (16-byte elements) of its sweep workspace
    size_t grad_off;        // offset (doubles) of its dT/d eps block (gradient only)
    // Schedule of its forward sweep (chosen per column size by the host's
    // tuning table; the gradient sweep ignores it):
    int8_t tc;              // 1: dense products on the tensor cores (RGF_MIXED_TC
                            // launches only), 0: on the FP32 / FP64 pipes
    int8_t panel;           // Gauss-Jordan panel width; 0 = the widest that fits
    int8_t pairs;           // 1: t I-bonded column pairs share one inverse
    int8_t sched_pad;
};

// The default schedule of a chain: everything on, the widest panel.
__host__ __device__ inline void default_sched(ChainDev& ch) {
    ch.tc = 1;
    ch.panel = 0;
    ch.pairs = 1;
    ch.sched_pad = 0;
}

// Number of 16-byte elements of the decimation workspace of one lead problem.
__host__ __device__ inline size_t lead_ws_elems(int N) {
    size_t KL = (size_t)col_KL(N);
    return KL * KL;   // the KL x KL (binary64) transverse mode basis, with room to spare
}
__host__ __device__ inline size_t lead_out_elems(int N) {
    size_t KL = (size_t)col_KL(N), KR = (size_t)col_KR(N);
    return 3 * (KL * KL + KR * KR) + KL;
}
// The sweep of one chain runs as two halves, one from each lead (see
// rgf_half.cuh).  Workspace of one half: X, G, P (each KL x KL) and one
// element holding the half's status flags; a chain holds two halves.
__host__ __device__ inline size_t half_ws_elems(int N) {
    size_t KL = (size_t)col_KL(N);
    return 3 * KL * KL + 1;
}
__host__ __device__ inline size_t sweep_ws_elems(int N) { return 2 * half_ws_elems(N); }
// With ndom > 2 domains per chain the ndom - 2 interior domains hold X, G, P
// and A (each KL x KL) and a flag element each, after the two halves.
__host__ __device__ inline size_t interior_ws_elems(int N) {
    size_t KL = (size_t)col_KL(N);
    return 4 * KL * KL + 1;
}
__host__ __device__ inline size_t chain_ws_elems(int N, int ndom) {
    return sweep_ws_elems(N) + (size_t)(ndom > 2 ? ndom - 2 : 0) * interior_ws_elems(N);
}
// First column of domain d of ndom over ncol columns (domain d covers columns
// dom_bound(d) .. dom_bound(d + 1) - 1; two domains split at ncol / 2).  The
// inner boundaries are even columns (c0 or c2 of a cell), so that an interior
// domain starts with a t I-bonded pair of columns; with ndom <= ncol / 2 every
// domain keeps two columns or more.
__host__ __device__ inline int dom_bound(int ncol, int d, int ndom) {
    return d >= ndom ? ncol : (int)((((long long)ncol * d) / ndom) & ~1ll);
}

// Shared memory of the sweep / lead kernels for a largest column size Kmax
// (tc: with the tensor-core area of the RGF_MIXED_TC path).
size_t sweep_smem_bytes(int Kmax, bool tc = false);
// Whether the tensor-core layout (the sweep's buffers beside the digit tiles)
// fits a block's shared memory for columns of up to Kmax orbitals: up to
// Kmax = 970 (N = 1940).  Wider chains of the _TC precisions run their
// products on the pipes.
bool tc_layout_fits(int Kmax);

// Controls of the decimation (process-wide, set through rgf_set_lead_controls):
// iteration cap and the tolerance of the fixed-point residual test.
struct LeadControls {
    int max_iter;
    double residual_tol;
};
LeadControls lead_controls();
void set_lead_controls(LeadControls c);

// Kernel launchers (return cudaGetLastError() after the launch).
// One block per lead problem computes both leads; lead_status / lead_iters
// hold [2 * nlead] entries (left, right per problem).
cudaError_t launch_lead(const LeadDev* leads, int nlead, int Kmax, double eta_lead,
                        void* ws, void* out, int* lead_status, int* lead_iters,
                        cudaStream_t st);

// The conductance of every chain in three launches on `st`:
//   launch_prep:  the lead-attached end column of each half in binary64, in the
//                 leads' transverse-mode basis (2 blocks per chain);
//   launch_half:  the column recursion of each domain (ndom blocks per chain:
//                 the two halves, and with ndom > 2 the interior domains);
//   launch_merge: the domains joined across their boundary bonds, and the
//                 trace (1 block per chain; writes T and status).
// leadout / lead_status as launch_lead left them; ws: chain_ws_elems per chain.
cudaError_t launch_prep(int precision, const ChainDev* chains, const int* order, int nchains,
                        int Kmax, double eta_device, const void* leadout, const int* lead_status,
                        const LeadDev* leads, void* ws, cudaStream_t st, int ndom = 2);
cudaError_t launch_half(int precision, const ChainDev* chains, const int* order, int nchains,
                        int Kmax, double eta_device, const void* leadout, const int* lead_status,
                        const LeadDev* leads, void* ws, cudaStream_t st, int ndom = 2);
cudaError_t launch_merge(int precision, const ChainDev* chains, const int* order, int nchains,
                         int Kmax, double eta_device, const void* leadout, const int* lead_status,
                         const LeadDev* leads, void* ws, double* T, int32_t* status,
                         cudaStream_t st, int ndom = 2);
// The domain kernels of ndom > 2 (rgf_domains.cu): launch_domains runs every
// domain of every chain (ndom blocks per chain); configure_domains sets their
// shared-memory limits.
cudaError_t launch_domains(int precision, const ChainDev* chains, const int* order, int nchains,
                           int Kmax, double eta_device, const void* leadout,
                           const int* lead_status, const LeadDev* leads, void* ws, int ndom,
                           cudaStream_t st);
cudaError_t configure_domains(int precision, int Kmax);
// The tree of joins that combines the ndom - 2 interior domains of every
// chain into one segment (ceil(log2(ndom - 2)) launches; nothing for ndom <=
// 3); launch_merge runs it before the final joins.
cudaError_t launch_tree(int precision, const ChainDev* chains, const int* order, int nchains,
                        int Kmax, double eta_device, const void* leadout, const int* lead_status,
                        const LeadDev* leads, void* ws, int ndom, cudaStream_t st);

// The same three steps as one persistent kernel (rgf_batch.cu): one block per
// SM (at most 2 * nchains), each taking the next half from a work queue in the
// order of `order` (item 2i + h = half h of chain order[i]), preparing its end
// column, running its recursion and, if it finishes second of its chain's two
// halves, joining them and writing T and status.  queue: batch_queue_ints(n)
// zeroed ints (the caller zeroes them before every launch); nsm: the number of
// persistent blocks.
inline size_t batch_queue_ints(int nchains) { return 1 + (size_t)nchains; }
cudaError_t launch_batch(int precision, const ChainDev* chains, const int* order, int nchains,
                         int Kmax, double eta_device, const void* leadout, const int* lead_status,
                         const LeadDev* leads, void* ws, double* T, int32_t* status, int* queue,
                         int nsm, cudaStream_t st);
// Sets the kernels' shared-memory limits for a largest column size Kmax (done by
// every launcher; also callable ahead of a stream capture): configure_sweep
// for all of them, configure_batch for the persistent kernel alone.
cudaError_t configure_sweep(int precision, int Kmax);
cudaError_t configure_batch(int precision, int Kmax);

// Two-sided sweep (rgf_grad.cu): workspace (16-byte elements) of one chain
// with segments of seg_cols columns, and the launcher (seg_cols: [nchains] on
// the device).  out_mode: OUT_GRAD writes dT/d eps into dT, OUT_LDOS the local
// density of states into rho (zero-initialised doubles, chain c's block at
// chains[c].grad_off; the unused pointer may be null).
enum : int { OUT_GRAD = 1, OUT_LDOS = 2 };
size_t grad_ws_elems(int N, int L, int seg_cols);
cudaError_t launch_grad(int precision, const ChainDev* chains, const int* order, int nchains,
                        int Kmax, double eta_device, const void* leadout, const int* lead_status,
                        const LeadDev* leads, void* ws, const int* seg_cols, double* T, double* dT,
                        double* rho, int out_mode, int32_t* status, cudaStream_t st);

}  // namespace rgf
