// Allocation-free entry point: the FP64 final reduction of one complex
// contraction, with its scratch in a file-scope device array.
//
// Some callers cannot allocate device memory: a host program whose device
// memory is all owned by another allocator (a framework's pool or a fixed
// per-process budget) may not call cudaMalloc behind that allocator's back,
// and code on a latency-critical path cannot afford the device-wide
// synchronisation a cudaMalloc/cudaFree may cause. tnc_contract needs a
// workspace for its partial sums (allocated by the library or handed in by
// the caller); tnc_reduce_pair_noalloc instead keeps them in the static array
// below, which every GPU that loads libtnc holds (1 MiB) until the process
// exits.
#include "tnc.h"

#include <mutex>
#include <string>

#include "kernels.h"

namespace {

constexpr int kMaxPartials = TNC_NOALLOC_MAX_PARTIALS;  // complex doubles
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double2 g_noalloc_scratch[kMaxPartials];

std::mutex g_mu;
double2* g_scratch_ptr[kMaxDevices] = {nullptr};


// Device address of the scratch array on the current device. In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached. The cache holds addresses
// in each device's primary context, the runtime's context; it is not valid
// in other driver contexts or after cudaDeviceReset.
cudaError_t scratch_for_current_device(double2** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double2*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" tnc_status tnc_reduce_pair_noalloc(const float* a_c64, const float* b_c64, int m_log2,
                                              int n_log2, int k_log2, double* out_c128, void* stream) {
    auto fail = [](tnc_status st, const std::string& m) {
        tnc::set_last_error(m);
        return st;
    };
    if (!a_c64 || !b_c64 || !out_c128) return fail(TNC_E_INVALID, "NULL pointer");
    if (m_log2 < 0 || n_log2 < 0 || k_log2 < 0) return fail(TNC_E_INVALID, "negative size");
    if (m_log2 + n_log2 > 6) return fail(TNC_E_INVALID, "M*N exceeds 64 outputs");
    if (k_log2 > 31) return fail(TNC_E_INVALID, "K exceeds 2^31");
    const int64_t K = 1ll << k_log2;
    int64_t chunks = K / 1024;
    if (chunks < 1) chunks = 1;
    if (chunks > 1024) chunks = 1024;
    const int64_t R = 1ll << (m_log2 + n_log2);
    if (chunks * R > kMaxPartials) return fail(TNC_E_INVALID, "partial sums exceed the static scratch");

    double2* scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return fail(TNC_E_CUDA, std::string("scratch lookup failed: ") + cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;
    // Row-major A[M][K] and B[K][N] as per-bit strides of the shared kernel.
    tnc::RootParams rp{};
    tnc::GemmParams& g = rp.g;
    g.A.ptr = reinterpret_cast<const float2*>(a_c64);
    g.B.ptr = reinterpret_cast<const float2*>(b_c64);
    g.mb = m_log2;
    g.nb = n_log2;
    g.kb = k_log2;
    for (int j = 0; j < m_log2; ++j) g.am[j] = K << j;
    for (int j = 0; j < k_log2; ++j) {
        g.ak[j] = 1ll << j;
        g.bk[j] = (1ll << n_log2) << j;
    }
    for (int j = 0; j < n_log2; ++j) g.bn[j] = 1ll << j;
    rp.chunks = (int)chunks;
    tnc::PermParams pp{};
    pp.obits = m_log2 + n_log2;
    for (int j = 0; j < pp.obits; ++j) pp.ostride[j] = 1ll << j;
    // every partial slot is written before it is read; only the output starts at zero
    e = cudaMemsetAsync(out_c128, 0, R * 16, s);
    if (e == cudaSuccess) e = tnc::launch_root_partials(rp, 1, scratch, s);
    if (e == cudaSuccess) e = tnc::launch_accumulate_partials(scratch, (int)chunks, pp,
                                                              reinterpret_cast<double2*>(out_c128), s);
    if (e != cudaSuccess) return fail(TNC_E_CUDA, std::string("launch failed: ") + cudaGetErrorString(e));
    return TNC_OK;
}
