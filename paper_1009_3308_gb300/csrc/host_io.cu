// RHS evaluations from host buffers (Eq. (ode) as sphnse_rhs), pipelined:
// call k copies alpha (and forcing) into device staging slot k mod 2 on an
// upload stream, evaluates F on the plan's stream, and returns F to the
// host.
//
// Direct output (out_h page-locked and mapped into the device's address
// space, the RHS on the fused tensor-core kernels): the call waits on the
// host for its upload, so the plan's stream carries nothing but the RHS
// kernels and every call overlaps its predecessor (programmatic dependent
// launch); the analysis writes F straight into out_h (NVLink-C2C on a Grace
// system) and its last CTA reports the call's completion in a mapped host
// flag, which sphnse_host_wait reads.  Before refilling a slot the call
// waits (host) for the RHS that read it.
//
// Otherwise F is copied back on a download stream: call k + 1's upload
// overlaps call k's RHS, and call k's download overlaps call k + 1's RHS.
// Slot reuse is ordered on the device: upload k waits for RHS k - 2 (which
// read the slot), and RHS k waits for download k - 2 (which read the slot's
// output).
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <thread>

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

// the device address of a page-locked, mapped host array (false otherwise)
bool mapped_address(const void* p, void** dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return false;
    *dev = at.devicePointer;
    return true;
}

int flag_init(HostIO& h) {
    if (h.flag) return SPHNSE_OK;
    void* f = nullptr;
    if (cudaHostAlloc(&f, sizeof(unsigned long long), cudaHostAllocMapped) != cudaSuccess) return SPHNSE_E_NOMEM;
    *static_cast<volatile unsigned long long*>(f) = 0ull;
    if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&h.dflag), f, 0) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&h.dcnt), sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(h.dcnt, 0, sizeof(unsigned)) != cudaSuccess) {
        cudaFreeHost(f);
        return SPHNSE_E_NOMEM;
    }
    h.flag = static_cast<volatile unsigned long long*>(f);
    return SPHNSE_OK;
}

// wait (host) until direct-output call `ticket` has written F
int flag_wait(HostIO& h, long long ticket) {
    const auto t0 = std::chrono::steady_clock::now();
    while (*h.flag < static_cast<unsigned long long>(ticket + 1)) {
        if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(30)) return SPHNSE_E_TIMEOUT;
        std::this_thread::yield();
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    return SPHNSE_OK;
}

}  // namespace

void host_io_free(sphnse_plan* P) {
    HostIO& h = P->hio;
    if (h.flag) cudaStreamSynchronize(P->stream);
    if (h.flag) cudaFreeHost(const_cast<unsigned long long*>(h.flag));
    if (h.dcnt) cudaFree(h.dcnt);
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
    // a direct-output call k - 2 read this slot outside the stream order
    if (k >= 2 && h.direct[s] == k - 2 && (rc = flag_wait(h, k - 2))) return rc;
    void* dout = nullptr;
    if (mapped_address(out_h, &dout) && tc_rhs_fused(P)) {
        if ((rc = flag_init(h))) return rc;
        if (k >= 2 && h.direct[s] != k - 2 && cudaEventSynchronize(h.ev_rhs[s]) != cudaSuccess) return SPHNSE_E_CUDA;
        if (cudaMemcpyAsync(h.din[s], alpha_h, b, cudaMemcpyHostToDevice, h.up) != cudaSuccess) return SPHNSE_E_CUDA;
        if (forcing_h && cudaMemcpyAsync(h.dfo[s], forcing_h, b, cudaMemcpyHostToDevice, h.up) != cudaSuccess)
            return SPHNSE_E_CUDA;
        if (cudaStreamSynchronize(h.up) != cudaSuccess) return SPHNSE_E_CUDA;
        P->done_cnt = h.dcnt;
        P->done_flag = h.dflag;
        P->done_ticket = static_cast<unsigned long long>(k + 1);
        rc = rhs_device(P, static_cast<const double*>(h.din[s]),
                        forcing_h ? static_cast<const double*>(h.dfo[s]) : nullptr, static_cast<double*>(dout));
        P->done_cnt = nullptr;
        P->done_flag = nullptr;
        if (rc) return rc;
        h.direct[s] = k;
        h.calls = k + 1;
        if (ticket) *ticket = k;
        return SPHNSE_OK;
    }
    const bool reuse = k >= 2 && h.direct[s] != k - 2;
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
    // direct output: the flag holds the last finished direct call's ticket + 1
    if (h.direct[ticket & 1] == ticket) return flag_wait(h, ticket);
    // the slot's event belongs to this ticket or a later call: either way
    // waiting on it covers the ticket
    if (cudaEventSynchronize(h.ev_down[ticket & 1]) != cudaSuccess) return SPHNSE_E_CUDA;
    return SPHNSE_OK;
}

}  // extern "C"
