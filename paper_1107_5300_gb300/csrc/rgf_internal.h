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
    size_t off;      // offset (in 16-byte complex elements) of this problem's
                     // Sigma_L [KL*KL], Sigma_R [KR*KR], Gamma_L [KL*KL], Gamma_R [KR*KR]
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
};

// Number of 16-byte elements of the decimation workspace of one lead problem.
inline size_t lead_ws_elems(int N) {
    size_t KL = (size_t)col_KL(N);
    return KL * KL;   // the KL x KL (binary64) transverse mode basis, with room to spare
}
inline size_t lead_out_elems(int N) {
    size_t KL = (size_t)col_KL(N), KR = (size_t)col_KR(N);
    return 2 * (KL * KL + KR * KR);
}
// Sweep workspace of one chain: X, G0, G1, P, Y (each KL x KL) and one
// element for the flag handed between the two blocks of a chain.
inline size_t sweep_ws_elems(int N) {
    size_t KL = (size_t)col_KL(N);
    return 5 * KL * KL + 1;
}

// Shared memory of the sweep / lead kernels for a largest column size Kmax
// (tc: with the tensor-core area of the RGF_MIXED_TC path).
size_t sweep_smem_bytes(int Kmax, bool tc = false);

// Kernel launchers (return cudaGetLastError() after the launch).
// One block per lead problem computes both leads; lead_status / lead_iters
// hold [2 * nlead] entries (left, right per problem).
cudaError_t launch_lead(const LeadDev* leads, int nlead, int Kmax, double eta_lead,
                        void* ws, void* out, int* lead_status, int* lead_iters,
                        cudaStream_t st);

cudaError_t launch_sweep(int precision, const ChainDev* chains, const int* order, int nchains,
                         int Kmax, double eta_device, const void* leadout, const int* lead_status,
                         const LeadDev* leads, void* ws, double* T, int32_t* status,
                         cudaStream_t st);

// Gradient sweep: workspace (16-byte elements) of one chain with segments of
// seg_cols columns, and the launcher (seg_cols: [nchains] on the device; dT:
// zero-initialised doubles, chain c's block at chains[c].grad_off).
size_t grad_ws_elems(int N, int L, int seg_cols);
cudaError_t launch_grad(int precision, const ChainDev* chains, const int* order, int nchains,
                        int Kmax, double eta_device, const void* leadout, const int* lead_status,
                        const LeadDev* leads, void* ws, const int* seg_cols, double* T, double* dT,
                        int32_t* status, cudaStream_t st);

}  // namespace rgf
