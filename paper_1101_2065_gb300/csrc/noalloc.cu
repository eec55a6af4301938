// Allocation-free variant of the Sigma_c grid evaluation (a7).
//
// Some callers cannot allocate device memory: an application whose device
// memory is owned entirely by another allocator (a framework's caching
// allocator or a serving engine that reserves its pool up front), or a
// latency-critical loop that must never wait on the driver's allocator.
// gw_sigma_c_static serves them: it needs a small scratch table of Cauchy
// kernel values, and keeps it in a fixed array compiled into this library
// instead of allocating it.  The caller passes the input and output device
// buffers.
//
// The scratch array exists once per GPU that loads the library and stays
// there until the process exits.  All calls on a device share it, so calls
// whose kernels overlap on the GPU (two host threads, or two streams) race
// on it; serialise them.  Each call rewrites every table entry it reads, so
// nothing left by an earlier call is used.  The first call in a CUDA context
// (normally the device's primary context) looks up the array's device
// address (cudaGetSymbolAddress) with that context current and caches it
// per context, so a device reset or another context on the same device
// gets its own lookup; make that first call before any stream capture.
#include <cuda.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "internal.h"

namespace {

// Largest table: n_sig + 2 n_omega - 1 complex entries (1 MiB per GPU).
constexpr long long kStaticTableMax = 1LL << 16;
static __device__ __align__(256) double2 g_sigc_table[kStaticTableMax];

std::mutex g_mutex;
std::vector<std::pair<CUcontext, double2*>> g_table_ptr;   // address of the table per CUDA context

// The calling thread's current CUDA context (driver entry point resolved
// through the runtime, so the library needs no link to libcuda).
CUcontext current_context() {
    typedef CUresult (*GetCurrent)(CUcontext*);
    static GetCurrent fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        fn = reinterpret_cast<GetCurrent>(p);
    }
    CUcontext c = nullptr;
    return fn(&c) == CUDA_SUCCESS ? c : nullptr;
}

__global__ void k_static_cauchy_table(double2* __restrict__ K, long long dmin, long long nd, double dw, double eta) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nd) return;
    double x = (double)(dmin + t) * dw;
    double den = x * x + eta * eta;
    K[t] = make_double2(x / den, -eta / den);
}

__global__ void __launch_bounds__(256) k_static_sigma_c(const double* __restrict__ sig, int n_sig, int j0, int N,
                                                        double dw, const double2* __restrict__ K, long long dmin,
                                                        int n_states, double2* __restrict__ out) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int nk = 2 * N - 1;
    if (t >= (long long)n_states * nk) return;
    int s = (int)(t / nk);
    int k = (int)(t % nk) - (N - 1);
    const double* sg = sig + (long long)s * n_sig;
    double re = 0.0, im = 0.0;
    for (int q = 0; q < n_sig; ++q) {
        int j = j0 + q;
        double2 kv = K[(long long)(k - j) - dmin];
        double v = sg[q];
        re = fma(v, kv.x, re);
        im = fma(v, j >= 0 ? kv.y : -kv.y, im);
    }
    out[t] = make_double2(dw * re, dw * im);
}

void set_msg(char* err, size_t len, const char* msg) {
    if (err && len) {
        std::strncpy(err, msg, len - 1);
        err[len - 1] = '\0';
    }
}

}  // namespace

extern "C" gw_status gw_sigma_c_static(const double* sigma, int n_states, int n_sig, int j0, int n_omega,
                                       double d_omega, double eta, double* sigc, void* stream, char* err,
                                       size_t err_len) {
    set_msg(err, err_len, "");
    if (!sigma || !sigc || n_states <= 0 || n_sig <= 0 || n_omega <= 0 || !(d_omega > 0.0) || !(eta > 0.0)) {
        set_msg(err, err_len, "gw_sigma_c_static: invalid argument");
        return GW_ERR_INVALID_ARG;
    }
    const long long nd = (long long)n_sig + 2LL * n_omega - 1;
    if (nd > kStaticTableMax) {
        char buf[160];
        std::snprintf(buf, sizeof(buf),
                      "gw_sigma_c_static: n_sig + 2 n_omega - 1 = %lld exceeds the static table of %lld entries",
                      nd, kStaticTableMax);
        set_msg(err, err_len, buf);
        return GW_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_msg(err, err_len, "gw_sigma_c_static: no usable current device");
        return GW_ERR_CUDA;
    }
    double2* table = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        CUcontext ctx = current_context();
        for (auto& kv : g_table_ptr)
            if (ctx && kv.first == ctx) table = kv.second;
        if (!table) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_sigc_table);     // also makes the runtime's context current
            if (e != cudaSuccess) {
                cudaGetLastError();
                set_msg(err, err_len, cudaGetErrorString(e));
                return GW_ERR_CUDA;
            }
            table = static_cast<double2*>(p);
            ctx = current_context();
            if (!ctx) {
                set_msg(err, err_len, "gw_sigma_c_static: no current CUDA context");
                return GW_ERR_CUDA;
            }
            g_table_ptr.emplace_back(ctx, table);
        }
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // d = k - j for k in [-(N-1), N-1] and j in [j0, j0 + n_sig - 1]
    const long long dmin = -(long long)(n_omega - 1) - (j0 + n_sig - 1);
    k_static_cauchy_table<<<(unsigned)((nd + 255) / 256), 256, 0, st>>>(table, dmin, nd, d_omega, eta);
    const long long tot = (long long)n_states * (2LL * n_omega - 1);
    k_static_sigma_c<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(sigma, n_sig, j0, n_omega, d_omega, table,
                                                                    dmin, n_states,
                                                                    reinterpret_cast<double2*>(sigc));
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_msg(err, err_len, cudaGetErrorString(e));
        return GW_ERR_CUDA;
    }
    return GW_OK;
}
