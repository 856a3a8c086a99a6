// Density-fitting object operations of the paper's section "Density fitting utilities", eqs. (1)-(3), on
// dense FP64 three-index tensors I[g][r][s] (g the auxiliary index) held on the device:
//   (1) index transformations of the first, second or auxiliary index by a matrix;
//   (2) contractions of two objects into a matrix over their second indices (summed over g and the first
//       index), a four-index matrix over both index pairs (summed over g), or a matrix over their
//       auxiliary indices (summed over both orbital indices);
//   (3) contractions with a density matrix into an auxiliary vector and back, and with a four-index
//       matrix G into a new object.
// Every operation is one FP64 GEMM over a reshaped view of the tensors (the first-index transformation one
// GEMM per auxiliary row), on the handle's stream.
#include <algorithm>
#include <climits>
#include <memory>

#include "common.cuh"

struct df_tensor {
    df_handle* h = nullptr;
    int naux = 0, nr = 0, ns = 0;
    dfhf::DevBuf<double> d;
    long long size() const { return (long long)naux * nr * ns; }
};

namespace dfhf {

namespace {

// C = op(A) op(B) with the rows of C in blocks small enough for the GEMM grid (rows of C: m)
void gemm_rows(cudaStream_t s, bool ta, bool tb, long long m, long long n, long long k, const double* A, long long lda,
               const double* B, long long ldb, double* C, long long ldc) {
    if (n > INT_MAX || k > INT_MAX || lda > INT_MAX || ldb > INT_MAX || ldc > INT_MAX)
        throw Error{DF_E_ARG, "density-fitting operation: a matrix dimension exceeds the GEMM's range"};
    const long long block = 65535LL * 64;
    for (long long r0 = 0; r0 < m; r0 += block) {
        const long long mr = std::min(block, m - r0);
        const double* Ab = ta ? A + r0 : A + r0 * lda;   // op(A) rows r0.. are columns of a stored-transposed A
        dgemm(s, ta, tb, (int)mr, (int)n, (int)k, 1.0, Ab, (int)lda, B, (int)ldb, 0.0, C + r0 * ldc, (int)ldc);
    }
}

df_tensor* new_tensor(df_handle* h, int naux, int nr, int ns) {
    if (naux < 1 || nr < 1 || ns < 1) throw Error{DF_E_ARG, "density-fitting object: every dimension must be >= 1"};
    df_tensor* t = new df_tensor();
    t->h = h;
    t->naux = naux;
    t->nr = nr;
    t->ns = ns;
    try {
        t->d.alloc((size_t)t->size());
    } catch (...) {
        delete t;
        throw;
    }
    return t;
}

// a host array on the device for the duration of one operation
void upload(df_handle* h, DevBuf<double>& buf, const double* host, long long count) {
    buf.alloc((size_t)count);
    DF_CUDA(cudaMemcpyAsync(buf.p, host, sizeof(double) * count, cudaMemcpyHostToDevice, h->stream));
}

void download(df_handle* h, double* host, const DevBuf<double>& buf, long long count) {
    DF_CUDA(cudaMemcpyAsync(host, buf.p, sizeof(double) * count, cudaMemcpyDeviceToHost, h->stream));
    DF_CUDA(cudaStreamSynchronize(h->stream));
}

template <typename F>
int guarded(df_handle* h, F&& body) {
    try {
        DF_CUDA(cudaSetDevice(h->device));
        body();
    } catch (const Error& e) {
        h->last_error = e.msg;
        return e.code;
    }
    return DF_OK;
}

}  // namespace
}  // namespace dfhf

using namespace dfhf;

extern "C" {

int df_tensor_create(df_handle* h, int naux, int nr, int ns, const double* host_init, df_tensor** out) {
    if (!h || !out) return DF_E_ARG;
    *out = nullptr;
    return guarded(h, [&] {
        std::unique_ptr<df_tensor> t(new_tensor(h, naux, nr, ns));
        if (host_init)
            DF_CUDA(cudaMemcpyAsync(t->d.p, host_init, sizeof(double) * t->size(), cudaMemcpyHostToDevice, h->stream));
        else
            t->d.zero(h->stream);
        DF_CUDA(cudaStreamSynchronize(h->stream));
        *out = t.release();
    });
}

int df_tensor_from_B(df_handle* h, df_tensor** out) {
    if (!h || !out) return DF_E_ARG;
    *out = nullptr;
    if (!h->built || !h->B.p) {
        h->last_error = "df_tensor_from_B: B not built";
        return DF_E_STATE;
    }
    return guarded(h, [&] {
        std::unique_ptr<df_tensor> t(new_tensor(h, h->naux, h->n, h->n));
        unpack_rows(h, h->B.p, 0, h->naux, t->d.p);
        DF_CUDA(cudaStreamSynchronize(h->stream));
        *out = t.release();
    });
}

int df_tensor_shape(const df_tensor* t, int* naux, int* nr, int* ns) {
    if (!t || !naux || !nr || !ns) return DF_E_ARG;
    *naux = t->naux;
    *nr = t->nr;
    *ns = t->ns;
    return DF_OK;
}

int df_tensor_get(const df_tensor* t, double* host) {
    if (!t || !host) return DF_E_ARG;
    return guarded(t->h, [&] { download(t->h, host, t->d, t->size()); });
}

void df_tensor_free(df_tensor* t) {
    if (!t) return;
    if (t->h && t->h->stream) cudaStreamSynchronize(t->h->stream);
    delete t;
}

int df_op_transform(const df_tensor* I, int which, const double* M, int m_rows, int m_cols, df_tensor** out) {
    if (!I || !M || !out || m_rows < 1 || m_cols < 1) return DF_E_ARG;
    *out = nullptr;
    df_handle* h = I->h;
    if ((which == 0 && m_rows != I->nr) || (which == 1 && m_rows != I->ns) || (which == 2 && m_cols != I->naux) ||
        which < 0 || which > 2) {
        h->last_error = "df_op_transform: M does not match the transformed index";
        return DF_E_ARG;
    }
    return guarded(h, [&] {
        cudaStream_t s = h->stream;
        DevBuf<double> dM;
        upload(h, dM, M, (long long)m_rows * m_cols);
        std::unique_ptr<df_tensor> t;
        if (which == 0) {
            // I'_{g,ts} = sum_r M_rt I_{g,rs}: per auxiliary row M^T (nt x nr) I_g (nr x ns)
            t.reset(new_tensor(h, I->naux, m_cols, I->ns));
            for (int g = 0; g < I->naux; ++g)
                gemm_rows(s, true, false, m_cols, I->ns, I->nr, dM.p, m_cols, I->d.p + (long long)g * I->nr * I->ns,
                          I->ns, t->d.p + (long long)g * m_cols * I->ns, I->ns);
        } else if (which == 1) {
            // I'_{g,rt} = sum_s I_{g,rs} M_st: (naux nr) x ns times ns x nt
            t.reset(new_tensor(h, I->naux, I->nr, m_cols));
            gemm_rows(s, false, false, (long long)I->naux * I->nr, m_cols, I->ns, I->d.p, I->ns, dM.p, m_cols, t->d.p,
                      m_cols);
        } else {
            // I'_{g,rs} = sum_d M'_gd I_{d,rs}: naux' x naux times naux x (nr ns)
            t.reset(new_tensor(h, m_rows, I->nr, I->ns));
            const long long rs = (long long)I->nr * I->ns;
            gemm_rows(s, false, false, m_rows, rs, I->naux, dM.p, I->naux, I->d.p, rs, t->d.p, rs);
        }
        DF_CUDA(cudaStreamSynchronize(s));   // dM is released on return
        *out = t.release();
    });
}

int df_op_contract(const df_tensor* I, const df_tensor* I2, int which, double* out) {
    if (!I || !I2 || !out || which < 0 || which > 2 || I->h != I2->h) return DF_E_ARG;
    df_handle* h = I->h;
    if ((which == 0 && (I2->naux != I->naux || I2->nr != I->nr)) || (which == 1 && I2->naux != I->naux) ||
        (which == 2 && (I2->nr != I->nr || I2->ns != I->ns))) {
        h->last_error = "df_op_contract: the objects' shared indices differ in length";
        return DF_E_ARG;
    }
    return guarded(h, [&] {
        cudaStream_t s = h->stream;
        DevBuf<double> R;
        long long count = 0;
        if (which == 0) {
            // M_st = sum_{g r} I_{g,rs} I2_{g,rt}: ((naux nr) x ns)^T times (naux nr) x nt
            count = (long long)I->ns * I2->ns;
            R.alloc((size_t)count);
            gemm_rows(s, true, false, I->ns, I2->ns, (long long)I->naux * I->nr, I->d.p, I->ns, I2->d.p, I2->ns, R.p,
                      I2->ns);
        } else if (which == 1) {
            // G_{rs,tu} = sum_g I_{g,rs} I2_{g,tu}: (naux x (nr ns))^T times naux x (nt nu)
            const long long rs = (long long)I->nr * I->ns, tu = (long long)I2->nr * I2->ns;
            count = rs * tu;
            R.alloc((size_t)count);
            gemm_rows(s, true, false, rs, tu, I->naux, I->d.p, rs, I2->d.p, tu, R.p, tu);
        } else {
            // M_gd = sum_rs I_{g,rs} I2_{d,rs}: naux x (nr ns) times (naux2 x (nr ns))^T
            const long long rs = (long long)I->nr * I->ns;
            count = (long long)I->naux * I2->naux;
            R.alloc((size_t)count);
            gemm_rows(s, false, true, I->naux, I2->naux, rs, I->d.p, rs, I2->d.p, rs, R.p, I2->naux);
        }
        download(h, out, R, count);
    });
}

int df_op_density_fit(const df_tensor* I, const double* M, double* D) {
    if (!I || !M || !D) return DF_E_ARG;
    df_handle* h = I->h;
    return guarded(h, [&] {
        // D_g = sum_rs I_{g,rs} M_rs: naux x (nr ns) times (nr ns) x 1
        const long long rs = (long long)I->nr * I->ns;
        DevBuf<double> dM, dD;
        upload(h, dM, M, rs);
        dD.alloc(I->naux);
        gemm_rows(h->stream, false, false, I->naux, 1, rs, I->d.p, rs, dM.p, 1, dD.p, 1);
        download(h, D, dD, I->naux);
    });
}

int df_op_density_back(const df_tensor* I, const double* D, double* M) {
    if (!I || !D || !M) return DF_E_ARG;
    df_handle* h = I->h;
    return guarded(h, [&] {
        // M_rs = sum_g D_g I_{g,rs}: 1 x naux times naux x (nr ns)
        const long long rs = (long long)I->nr * I->ns;
        DevBuf<double> dD, dM;
        upload(h, dD, D, I->naux);
        dM.alloc((size_t)rs);
        gemm_rows(h->stream, false, false, 1, rs, I->naux, dD.p, I->naux, I->d.p, rs, dM.p, rs);
        download(h, M, dM, rs);
    });
}

int df_op_apply_four_index(const df_tensor* I, const double* G, int nt, int nu, df_tensor** out) {
    if (!I || !G || !out || nt < 1 || nu < 1) return DF_E_ARG;
    *out = nullptr;
    df_handle* h = I->h;
    return guarded(h, [&] {
        // I'_{g,tu} = sum_rs I_{g,rs} G_{rs,tu}: naux x (nr ns) times (nr ns) x (nt nu)
        const long long rs = (long long)I->nr * I->ns, tu = (long long)nt * nu;
        DevBuf<double> dG;
        upload(h, dG, G, rs * tu);
        std::unique_ptr<df_tensor> t(new_tensor(h, I->naux, nt, nu));
        gemm_rows(h->stream, false, false, I->naux, tu, rs, I->d.p, rs, dG.p, tu, t->d.p, tu);
        DF_CUDA(cudaStreamSynchronize(h->stream));   // dG is released on return
        *out = t.release();
    });
}

}  // extern "C"
