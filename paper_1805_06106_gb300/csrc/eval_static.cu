// qbx_eval_noalloc: qbx_eval for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at evaluation time: real-time loops whose memory
// budget is fixed up front, or hosts whose allocator owns the whole device and forbids
// outside allocations.  This entry point computes what qbx_eval computes in QBX_FP64 (the
// same stages and formulas; the box-expansion passes run the library's per-warp kernels,
// so results agree with qbx_eval to rounding, about 1e-15 relative), but takes every
// piece of scratch from one fixed, file-scope device array of QBX_NOALLOC_SCRATCH_BYTES
// (48 MiB) that is part of the library image: every GPU that loads the library holds it
// until the process exits.
#include <mutex>

#include "qbx_internal.cuh"

namespace qbx {
size_t fixed_workspace_bytes(const qbx_tree *T, const qbx_eval_opts *o);
void eval_fixed(const qbx_tree *T, const qbx_lists *L, unsigned char *base, size_t cap, const double *w,
                const double *sigma, const double *mu, const double *nrm, const int *tgt_ctr,
                const qbx_eval_opts *o, double *pot, cudaStream_t st);
void set_error(const std::string &msg);
}  // namespace qbx

static __device__ __align__(256) unsigned char g_noalloc_scratch[QBX_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char *g_addr[MAX_DEVICES] = {};

// Device address of the scratch array for the current device.  In host code the array's
// name stands for a host-side shadow, not a device address, so it is looked up once per
// device with that device current.
unsigned char *scratch_on_current_device()
{
    int dev = -1;
    QBX_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) throw qbx::Error{QBX_ERR_INVALID_ARG, "device index out of range"};
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        QBX_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    return g_addr[dev];
}

}  // namespace

extern "C" int qbx_eval_noalloc(const qbx_tree *T, const qbx_lists *L, const double *w, const double *sigma,
                                const double *mu, const double *nrm, const int32_t *tgt_ctr,
                                const qbx_eval_opts *o, double *pot, void *stream)
{
    try {
        qbx::set_error("");
        qbx::check_eval_args(T, L, w, mu, nrm, tgt_ctr, o, pot);
        if (o->precision != QBX_FP64)
            throw qbx::Error{QBX_ERR_INVALID_ARG, "qbx_eval_noalloc evaluates in QBX_FP64 only"};
        size_t need = qbx::fixed_workspace_bytes(T, o);
        if (need > (size_t)QBX_NOALLOC_SCRATCH_BYTES)
            throw qbx::Error{QBX_ERR_INVALID_ARG, "problem needs " + std::to_string(need) +
                                                      " bytes of scratch; qbx_eval_noalloc holds " +
                                                      std::to_string((size_t)QBX_NOALLOC_SCRATCH_BYTES) +
                                                      " (use qbx_eval)"};
        unsigned char *base = scratch_on_current_device();
        qbx::eval_fixed(T, L, base, (size_t)QBX_NOALLOC_SCRATCH_BYTES, w, sigma, mu, nrm, tgt_ctr, o, pot,
                        (cudaStream_t)stream);
        return QBX_OK;
    } catch (const qbx::Error &e) {
        qbx::set_error(e.msg);
        return e.code;
    } catch (...) {
        qbx::set_error("unexpected exception");
        return QBX_ERR_CUDA;
    }
}
