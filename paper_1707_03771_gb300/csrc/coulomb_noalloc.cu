// df_coulomb_noalloc: the Coulomb matrix J = sum_P gamma_P B_P (gamma_P = sum B_{P,mu nu} D_{mu nu})
// for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: a host application that owns every byte of device memory
// through its own allocator and forbids libraries from allocating, or a latency-critical loop
// where an allocation (which may synchronise the device or fail under memory pressure) is not
// acceptable. For them this entry point runs the same Coulomb kernels as df_jk, but takes its
// scratch from one fixed array compiled into the library instead of from the handle's lazily
// allocated buffers. The caller still provides D and J (device memory), and the handle must hold B.
//
// The scratch array (48 MiB) is part of the library image: every GPU that loads the library holds
// it until the process exits. Every call shares it, so calls that overlap on the GPU (on different
// streams or from different host threads without ordering) race and give wrong results; calls on
// one stream are ordered and safe. The array keeps the last call's contents; each call writes every
// element it reads before reading it, so no clearing is needed.
#include <mutex>

#include "common.cuh"

namespace dfhf {
void coulomb_with_scratch(cudaStream_t s, const double* B, const Packing& pk, int naux, int n, const double* dD,
                          double* dJ, double* Dw, double* gamma, double* Jp);
}

namespace {

constexpr long long kScratchDoubles = 6291456;   // 48 MiB
static __device__ __align__(256) double g_coulomb_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device. In host code the array's name is only
// a host-side stand-in (passing it to a kernel would fault or silently touch the wrong memory), so
// the real address is looked up once per device with that device current and cached.
int scratch_address(int dev, double** out) {
    if (dev < 0 || dev >= kMaxDevices) return DF_E_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_coulomb_scratch);
        if (e != cudaSuccess || !p) return DF_E_CUDA;
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return DF_OK;
}

}  // namespace

extern "C" int df_coulomb_noalloc(df_handle* h, const double* D, double* J) {
    using namespace dfhf;
    if (!h || !D || !J) return DF_E_ARG;
    const long long row = h->pk.row;
    const long long gamma_len = ((long long)h->naux + 31) / 32 * 32;   // keeps Jp 256-byte aligned
    const long long need = 2 * row + gamma_len;
    if (need > kScratchDoubles) {
        h->last_error = "df_coulomb_noalloc: this system needs " + std::to_string(need) +
                        " doubles of scratch (2 packed rows + naux), more than the static maximum of " +
                        std::to_string(kScratchDoubles) + " (48 MiB); use df_jk";
        return DF_E_ARG;
    }
    if (!h->built || !h->B.p) {
        h->last_error = "df_coulomb_noalloc: B not built (call df_build_B first)";
        return DF_E_STATE;
    }
    if (cudaSetDevice(h->device) != cudaSuccess) return DF_E_CUDA;
    double* base = nullptr;
    int rc = scratch_address(h->device, &base);
    if (rc != DF_OK) {
        h->last_error = "df_coulomb_noalloc: cudaGetSymbolAddress failed";
        return rc;
    }
    try {
        coulomb_with_scratch(h->stream, h->B.p, h->pk, h->naux, h->n, D, J, base, base + row, base + row + gamma_len);
    } catch (const Error& e) {
        h->last_error = e.msg;
        return e.code;
    }
    return DF_OK;
}
