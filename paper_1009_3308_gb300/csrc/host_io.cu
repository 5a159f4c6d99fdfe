// RHS evaluations from host buffers (Eq. (ode) as sphnse_rhs), pipelined:
// call k copies alpha (and forcing) into device staging slot k mod 2 on an
// upload stream, evaluates F on the plan's stream, and copies F back on a
// download stream.  Call k + 1's upload overlaps call k's RHS, and call k's
// download overlaps call k + 1's RHS.  Slot reuse is ordered on the device:
// upload k waits for RHS k - 2 (which read the slot), and RHS k waits for
// download k - 2 (which read the slot's output).
#include <cuda_runtime.h>

#include "internal.h"

namespace sph {
namespace {

int host_io_init(sphnse_plan* P) {
    HostIO& h = P->hio;
    if (h.ready) return SPHNSE_OK;
    const size_t b = size_t(P->n_coeff) * 16;
    for (int s = 0; s < 2; ++s) {
        if (cudaMalloc(&h.din[s], b) != cudaSuccess || cudaMalloc(&h.dfo[s], b) != cudaSuccess ||
            cudaMalloc(&h.dout[s], b) != cudaSuccess)
            return SPHNSE_E_NOMEM;
        if (cudaEventCreateWithFlags(&h.ev_up[s], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h.ev_rhs[s], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h.ev_down[s], cudaEventDisableTiming) != cudaSuccess)
            return SPHNSE_E_CUDA;
    }
    if (cudaStreamCreateWithFlags(&h.up, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h.down, cudaStreamNonBlocking) != cudaSuccess)
        return SPHNSE_E_CUDA;
    h.ready = true;
    return SPHNSE_OK;
}

}  // namespace

void host_io_free(sphnse_plan* P) {
    HostIO& h = P->hio;
    if (h.up) cudaStreamSynchronize(h.up);
    if (h.down) cudaStreamSynchronize(h.down);
    for (int s = 0; s < 2; ++s) {
        for (void* q : {h.din[s], h.dfo[s], h.dout[s]})
            if (q) cudaFree(q);
        for (cudaEvent_t e : {h.ev_up[s], h.ev_rhs[s], h.ev_down[s]})
            if (e) cudaEventDestroy(e);
    }
    if (h.up) cudaStreamDestroy(h.up);
    if (h.down) cudaStreamDestroy(h.down);
    h = HostIO();
}

}  // namespace sph

using namespace sph;

extern "C" {

int sphnse_rhs_host(sphnse_plan* P, double t, const double* alpha_h, const double* forcing_h, double* out_h,
                    long long* ticket) {
    (void)t;
    if (!P || !alpha_h || !out_h) return SPHNSE_E_ARG;
    int rc = host_io_init(P);
    if (rc) return rc;
    HostIO& h = P->hio;
    const long long k = h.calls;
    const int s = int(k & 1);
    const size_t b = size_t(P->n_coeff) * 16;
    const bool reuse = k >= 2;
    // upload (after RHS k - 2 has read this slot)
    if (reuse && cudaStreamWaitEvent(h.up, h.ev_rhs[s], 0) != cudaSuccess) return SPHNSE_E_CUDA;
    if (cudaMemcpyAsync(h.din[s], alpha_h, b, cudaMemcpyHostToDevice, h.up) != cudaSuccess) return SPHNSE_E_CUDA;
    if (forcing_h && cudaMemcpyAsync(h.dfo[s], forcing_h, b, cudaMemcpyHostToDevice, h.up) != cudaSuccess)
        return SPHNSE_E_CUDA;
    if (cudaEventRecord(h.ev_up[s], h.up) != cudaSuccess) return SPHNSE_E_CUDA;
    // RHS on the plan's stream (after the upload, and after download k - 2 has read the output slot)
    if (cudaStreamWaitEvent(P->stream, h.ev_up[s], 0) != cudaSuccess) return SPHNSE_E_CUDA;
    if (reuse && cudaStreamWaitEvent(P->stream, h.ev_down[s], 0) != cudaSuccess) return SPHNSE_E_CUDA;
    if ((rc = rhs_device(P, static_cast<const double*>(h.din[s]),
                         forcing_h ? static_cast<const double*>(h.dfo[s]) : nullptr, static_cast<double*>(h.dout[s]))))
        return rc;
    if (cudaEventRecord(h.ev_rhs[s], P->stream) != cudaSuccess) return SPHNSE_E_CUDA;
    // download
    if (cudaStreamWaitEvent(h.down, h.ev_rhs[s], 0) != cudaSuccess) return SPHNSE_E_CUDA;
    if (cudaMemcpyAsync(out_h, h.dout[s], b, cudaMemcpyDeviceToHost, h.down) != cudaSuccess) return SPHNSE_E_CUDA;
    if (cudaEventRecord(h.ev_down[s], h.down) != cudaSuccess) return SPHNSE_E_CUDA;
    h.calls = k + 1;
    if (ticket) *ticket = k;
    return SPHNSE_OK;
}

int sphnse_host_wait(sphnse_plan* P, long long ticket) {
    if (!P || ticket < 0) return SPHNSE_E_ARG;
    HostIO& h = P->hio;
    if (!h.ready || ticket >= h.calls) return SPHNSE_E_ARG;
    // the slot's event belongs to this ticket or a later call: either way
    // waiting on it covers the ticket
    if (cudaEventSynchronize(h.ev_down[ticket & 1]) != cudaSuccess) return SPHNSE_E_CUDA;
    return SPHNSE_OK;
}

}  // extern "C"
