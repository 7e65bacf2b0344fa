// od_comm.cu -- communication endpoints of libod's inter-process transport.
//
// The paper's intra-node, inter-process path (Sec. IV, transport item 2):
// every process allocates one device communication buffer and a pool of
// interprocess events once, and every peer maps them through their IPC
// handles, so no handle is opened per message.  A face then moves by two
// device-to-device copies: the sender's boundary layer into its own buffer
// (od_face_copy export) followed by a recorded event, and -- after a host
// control message carrying the buffer offset and the event index -- the
// receiver's wait on that event and its copy from the mapped buffer into its
// ghost layer (od_face_copy import).  This file only owns the buffer, the
// events and their handles; the protocol runs in the caller.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

#include "od.h"

namespace od {
od_status set_last_error(od_status s, const std::string &msg);
}

static_assert(sizeof(cudaIpcMemHandle_t) == 64, "IPC memory handle size");
static_assert(sizeof(cudaIpcEventHandle_t) == 64, "IPC event handle size");

struct od_comm {
    int device = 0;
    bool opened = false;            // a peer's endpoint mapped into this process
    double *buf = nullptr;
    uint64_t bytes = 0;
    std::vector<cudaEvent_t> ev;
};

namespace {

constexpr uint32_t kMagic = 0x4d43444fu;  // "ODCM"

od_status fail(od_status s, const std::string &m) { return od::set_last_error(s, m); }
od_status cuda_fail(cudaError_t e, const char *what) {
    cudaGetLastError();
    return fail(OD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void destroy(od_comm *c) {
    if (!c) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    for (auto e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->buf) {
        if (c->opened) cudaIpcCloseMemHandle(c->buf);
        else cudaFree(c->buf);
    }
    if (prev >= 0) cudaSetDevice(prev);
    delete c;
}

}  // namespace

extern "C" {

OD_API od_status od_comm_create(od_comm **out, int32_t device, uint64_t bytes, int32_t nevents) {
    if (!out || bytes == 0 || bytes > ((uint64_t)1 << 40) || nevents < 1 || nevents > 4096)
        return fail(OD_EINVAL, "od_comm_create: bytes in [1, 2^40], nevents in [1, 4096]");
    *out = nullptr;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    od_comm *c = new od_comm();
    c->device = device;
    c->bytes = bytes;
    if ((e = cudaMalloc(&c->buf, bytes)) != cudaSuccess) {
        c->buf = nullptr;
        destroy(c);
        return fail(OD_ENOMEM, "od_comm_create: cannot allocate the communication buffer");
    }
    c->ev.assign((size_t)nevents, nullptr);
    for (auto &x : c->ev)
        if ((e = cudaEventCreateWithFlags(&x, cudaEventInterprocess | cudaEventDisableTiming)) != cudaSuccess) {
            x = nullptr;
            destroy(c);
            return cuda_fail(e, "cudaEventCreateWithFlags(interprocess)");
        }
    *out = c;
    return OD_OK;
}

OD_API od_status od_comm_handles(const od_comm *c, void *handles, uint64_t capacity) {
    if (!c || !handles) return fail(OD_EINVAL, "null argument");
    if (c->opened) return fail(OD_ESTATE, "od_comm_handles: only the owning process exports handles");
    const uint64_t need = OD_COMM_HANDLE_BYTES((uint64_t)c->ev.size());
    if (capacity < need) return fail(OD_EINVAL, "od_comm_handles: capacity below OD_COMM_HANDLE_BYTES(nevents)");
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    unsigned char *h = static_cast<unsigned char *>(handles);
    const uint32_t magic = kMagic, n = (uint32_t)c->ev.size();
    memcpy(h, &magic, 4);
    memcpy(h + 4, &n, 4);
    memcpy(h + 8, &c->bytes, 8);
    cudaIpcMemHandle_t mh;
    cudaError_t e = cudaIpcGetMemHandle(&mh, c->buf);
    if (e == cudaSuccess) memcpy(h + 16, &mh, 64);
    for (uint32_t i = 0; i < n && e == cudaSuccess; ++i) {
        cudaIpcEventHandle_t eh;
        e = cudaIpcGetEventHandle(&eh, c->ev[i]);
        if (e == cudaSuccess) memcpy(h + 80 + 64 * (size_t)i, &eh, 64);
    }
    if (prev >= 0) cudaSetDevice(prev);
    return e == cudaSuccess ? OD_OK : cuda_fail(e, "cudaIpcGet*Handle");
}

OD_API od_status od_comm_open(od_comm **out, int32_t device, const void *handles, uint64_t size) {
    if (!out || !handles || size < 16) return fail(OD_EINVAL, "null argument or short handle block");
    *out = nullptr;
    const unsigned char *h = static_cast<const unsigned char *>(handles);
    uint32_t magic = 0, n = 0;
    uint64_t bytes = 0;
    memcpy(&magic, h, 4);
    memcpy(&n, h + 4, 4);
    memcpy(&bytes, h + 8, 8);
    if (magic != kMagic || n < 1 || n > 4096 || size < OD_COMM_HANDLE_BYTES((uint64_t)n))
        return fail(OD_EINVAL, "od_comm_open: not an endpoint handle block");
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    od_comm *c = new od_comm();
    c->device = device;
    c->opened = true;
    c->bytes = bytes;
    cudaIpcMemHandle_t mh;
    memcpy(&mh, h + 16, 64);
    void *p = nullptr;
    if ((e = cudaIpcOpenMemHandle(&p, mh, cudaIpcMemLazyEnablePeerAccess)) != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaIpcOpenMemHandle (the endpoint of another process on this node)");
    }
    c->buf = static_cast<double *>(p);
    c->ev.assign(n, nullptr);
    for (uint32_t i = 0; i < n; ++i) {
        cudaIpcEventHandle_t eh;
        memcpy(&eh, h + 80 + 64 * (size_t)i, 64);
        if ((e = cudaIpcOpenEventHandle(&c->ev[i], eh)) != cudaSuccess) {
            c->ev[i] = nullptr;
            destroy(c);
            return cuda_fail(e, "cudaIpcOpenEventHandle");
        }
    }
    *out = c;
    return OD_OK;
}

OD_API od_status od_comm_buffer(const od_comm *c, double **buf, uint64_t *bytes, int32_t *nevents) {
    if (!c) return fail(OD_EINVAL, "null endpoint");
    if (buf) *buf = c->buf;
    if (bytes) *bytes = c->bytes;
    if (nevents) *nevents = (int32_t)c->ev.size();
    return OD_OK;
}

OD_API od_status od_comm_record(od_comm *c, int32_t event, void *stream) {
    if (!c || event < 0 || event >= (int32_t)c->ev.size()) return fail(OD_EINVAL, "od_comm_record: bad event");
    const cudaError_t e = cudaEventRecord(c->ev[(size_t)event], static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? OD_OK : cuda_fail(e, "cudaEventRecord");
}

OD_API od_status od_comm_wait(od_comm *c, int32_t event, void *stream) {
    if (!c || event < 0 || event >= (int32_t)c->ev.size()) return fail(OD_EINVAL, "od_comm_wait: bad event");
    const cudaError_t e = cudaStreamWaitEvent(static_cast<cudaStream_t>(stream), c->ev[(size_t)event], 0);
    return e == cudaSuccess ? OD_OK : cuda_fail(e, "cudaStreamWaitEvent");
}

OD_API od_status od_comm_destroy(od_comm *c) {
    destroy(c);
    return OD_OK;
}

}  // extern "C"
