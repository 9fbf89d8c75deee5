// rgf_tcgemm.cu -- rgf_zgemm_tc: the tensor-core complex product of the RGF
// step (rgf_tc.cuh) as a stand-alone entry point, C = A B for binary64
// complex matrices in device memory, sliced from binary64 (binary64-class
// accuracy, normwise).  One 512-thread block per 128 rows of C.
#include <cuda_runtime.h>

#include <string>

#include "rgf.h"
#include "rgf_tc.cuh"

namespace rgf {

void set_last_error(const std::string& msg);

namespace {

// Accessors of the binary64 operands (sliced from binary64) and of the
// output (the binary64 sum of the groups of 96 inner entries).
struct Z64Op {
    static constexpr bool kF64 = true;
    const zd* A;
    int lda;
    const zd* B;
    int ldb;
    zd* C;
    int ldc;
    int m0;
    __device__ zd a(int m, int k) const { return A[(size_t)(m0 + m) * lda + k]; }
    __device__ zd b(int k, int n) const { return B[(size_t)k * ldb + n]; }
    using Old = zd;
    __device__ bool colA() const { return false; }
    __device__ zd load(int m, int n, bool first) const {
        return first ? zd{0.0, 0.0} : C[(size_t)(m0 + m) * ldc + n];
    }
    __device__ void store(int m, int n, zd old, double re, double im, bool first) const {
        const zd x = {re, im};
        C[(size_t)(m0 + m) * ldc + n] = first ? x : cadd(old, x);
    }
};

// Dynamic shared memory of the kernel: the tensor-core area, raised so that
// only one block fits on an SM (each block holds all 512 TMEM columns).
constexpr size_t kSmem = tc::smem_bytes() > 120 * 1024 ? tc::smem_bytes() : 120 * 1024;

__global__ void __launch_bounds__(NT, 1)
zgemm_tc_kernel(int m, int n, int k, const zd* __restrict__ A, int lda, const zd* __restrict__ B,
                int ldb, zd* __restrict__ C, int ldc, int* __restrict__ err, long long wait_limit,
                int skip_commit) {
    const tc::Area ar{0};
    uint32_t phase = tc::setup(ar, wait_limit, skip_commit);
    const Z64Op op{A, lda, B, ldb, C, ldc, (int)blockIdx.x * 128};
    phase = tc::zgemm(op, min(128, m - op.m0), n, k, ar, phase);
    if (threadIdx.x == 0 && *(volatile int*)ar.err()) atomicExch(err, 1);
    tc::teardown(ar);
}

}  // namespace
}  // namespace rgf

namespace rgf {
namespace {

// One product on `st`, waited for; the kernel's completion-wait limit and the
// self-test switch are passed through.
rgf_status zgemm_tc_run(int m, int n, int k, const double* A, int lda, const double* B, int ldb,
                        double* C, int ldc, cudaStream_t st, long long wait_limit, int skip_commit) {
    int* derr = nullptr;
    int herr = 0;
    cudaError_t e = cudaMallocAsync(&derr, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(zgemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmem);
    if (e == cudaSuccess) {
        zgemm_tc_kernel<<<(m + 127) / 128, NT, kSmem, st>>>(m, n, k, (const zd*)A, lda,
                                                            (const zd*)B, ldb, (zd*)C, ldc, derr,
                                                            wait_limit, skip_commit);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (derr) {
        cudaError_t f = cudaFreeAsync(derr, st);
        if (e == cudaSuccess) e = f;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_last_error(std::string("rgf_zgemm_tc: ") + cudaGetErrorString(e));
        return RGF_ECUDA;
    }
    if (herr) {
        set_last_error("rgf_zgemm_tc: a tensor-core completion wait gave up");
        return RGF_ETIMEOUT;
    }
    return RGF_OK;
}

}  // namespace
}  // namespace rgf

extern "C" rgf_status rgf_zgemm_tc(int m, int n, int k, const double* A, int lda, const double* B,
                                   int ldb, double* C, int ldc, void* stream) {
    using namespace rgf;
    if (m < 0 || n < 0 || k < 0 || lda < (k > 0 ? k : 1) || ldb < (n > 0 ? n : 1) ||
        ldc < (n > 0 ? n : 1) || (m > 0 && n > 0 && (!C || (k > 0 && (!A || !B))))) {
        set_last_error("rgf_zgemm_tc: bad sizes or NULL pointer");
        return RGF_EINVAL;
    }
    if (m == 0 || n == 0) return RGF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (k == 0) {
        cudaError_t e = cudaMemset2DAsync(C, (size_t)ldc * 16, 0, (size_t)n * 16, (size_t)m, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_last_error(std::string("rgf_zgemm_tc: ") + cudaGetErrorString(e));
            return RGF_ECUDA;
        }
        return RGF_OK;
    }
    return zgemm_tc_run(m, n, k, A, lda, B, ldb, C, ldc, st, tc::kWaitLimit, 0);
}

extern "C" rgf_status rgf_zgemm_tc_selftest_timeout(void) {
    using namespace rgf;
    const int n = 64;
    double* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, 3 * (size_t)n * n * 16);
    if (e != cudaSuccess) {
        set_last_error(std::string("rgf_zgemm_tc_selftest_timeout: ") + cudaGetErrorString(e));
        return RGF_ECUDA;
    }
    e = cudaMemset(buf, 0, 3 * (size_t)n * n * 16);
    rgf_status s = RGF_ECUDA;
    if (e == cudaSuccess)
        s = zgemm_tc_run(n, n, n, buf, n, buf + 2 * n * n, n, buf + 4 * n * n, n, 0,
                         1000000ll /* about 0.5 ms of device clock */, 1);
    cudaFree(buf);
    return s;
}
