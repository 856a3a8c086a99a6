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
// it until the process exits. Its device address is resolved by df_init, with the handle's device
// current, and kept in the handle: under lazy module loading that lookup is what loads the module
// holding the array and commits its memory, so it happens when the handle is created and
// df_coulomb_noalloc itself allocates nothing. Every call shares the array, so calls that overlap on
// the GPU (on different streams or from different host threads without ordering) race and give wrong
// results; calls on one stream are ordered and safe. The array keeps the last call's contents; each
// call writes every element it reads before reading it, so no clearing is needed.
#include "common.cuh"

namespace dfhf {
void coulomb_with_scratch(cudaStream_t s, const double* B, const Packing& pk, int naux, int n, const double* dD,
                          double* dJ, double* Dw, double* gamma, double* Jp);

namespace {
constexpr long long kScratchDoubles = 6291456;   // 48 MiB
static __device__ __align__(256) double g_coulomb_scratch[kScratchDoubles];
}  // namespace

// Device address of the scratch array on the current device. In host code the array's name is only a
// host-side stand-in (passing it to a kernel would fault or silently touch the wrong memory), so the
// real address is asked of the runtime with the device current.
int noalloc_scratch_address(double** out, std::string* why) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_coulomb_scratch);
    if (e != cudaSuccess || !p) {
        if (why) *why = std::string("cudaGetSymbolAddress of the static scratch failed: ") + cudaGetErrorString(e);
        cudaGetLastError();   // the failure is reported here, not left for the next launch check
        return e == cudaErrorMemoryAllocation ? DF_E_NOMEM : DF_E_CUDA;
    }
    *out = static_cast<double*>(p);
    return DF_OK;
}

}  // namespace dfhf

extern "C" int df_coulomb_noalloc(df_handle* h, const double* D, double* J) {
    using namespace dfhf;
    if (!h) return DF_E_ARG;
    if (!D || !J) {
        h->last_error = "df_coulomb_noalloc: D and J must be device pointers, not null";
        return DF_E_ARG;
    }
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
    if (!h->noalloc_scratch) {
        h->last_error = "df_coulomb_noalloc: the static scratch was not available when the handle was created (" +
                        h->noalloc_error + ")";
        return DF_E_STATE;
    }
    const cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) {
        h->last_error = std::string("df_coulomb_noalloc: cudaSetDevice failed: ") + cudaGetErrorString(e);
        return DF_E_CUDA;
    }
    double* base = h->noalloc_scratch;
    try {
        coulomb_with_scratch(h->stream, h->B.p, h->pk, h->naux, h->n, D, J, base, base + row, base + row + gamma_len);
    } catch (const Error& err) {
        h->last_error = err.msg;
        return err.code;
    }
    return DF_OK;
}
