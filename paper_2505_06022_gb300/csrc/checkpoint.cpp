// Checkpoint and resume of a leapfrog simulation: the two time levels the
// recurrence needs (u^{n-1}, u^n) and the step count n, in a file with a fixed
// header.  The queue's stream is synchronised, so the fields hold the results of
// all work issued before the call.  Rows are stored without their pitch padding,
// so a checkpoint loads into any pitch.
#include <cstdio>
#include <cstring>
#include <vector>

#include "sy_internal.h"

namespace sy {
namespace {

constexpr int32_t kMagic = 0x53594331;  // "SYC1"

struct Header {
    int32_t magic;
    int32_t dtype;
    int32_t radius;
    int32_t reserved;
    int64_t ny, nx, step;
    float c2;
    int32_t pad;
};

sy_status copy_rows(Queue* q, const sy_stencil_params* p, const void* dev, std::vector<unsigned char>* host) {
    const size_t es = dtype_size(p->dtype), row = static_cast<size_t>(p->nx) * es;
    host->resize(row * static_cast<size_t>(p->ny));
    if (host->empty()) return SY_OK;
    SY_CUDA(cudaMemcpy2DAsync(host->data(), row, dev, static_cast<size_t>(p->pitch) * es, row,
                              static_cast<size_t>(p->ny), cudaMemcpyDeviceToHost, q->stream));
    SY_CUDA(cudaStreamSynchronize(q->stream));
    return SY_OK;
}

}  // namespace
}  // namespace sy

using namespace sy;

extern "C" {

sy_status sy_checkpoint_save(sy_queue_t qh, const char* path, const sy_stencil_params* p, const void* u_prev,
                             const void* u_cur, int64_t step) {
    clear_error();
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(stencil_param_checks(p));
    if (!path || !u_prev || !u_cur) return fail(SY_ERR_NULL_POINTER, "path or field pointer is NULL");
    SY_TRY(use_device(q));
    std::vector<unsigned char> a, b;
    SY_TRY(copy_rows(q, p, u_prev, &a));
    SY_TRY(copy_rows(q, p, u_cur, &b));
    Header h;
    std::memset(&h, 0, sizeof h);
    h.magic = kMagic;
    h.dtype = p->dtype;
    h.radius = p->radius;
    h.ny = p->ny;
    h.nx = p->nx;
    h.step = step;
    h.c2 = p->c2;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(SY_ERR_IO, "cannot open %s for writing", path);
    bool ok = std::fwrite(&h, sizeof h, 1, f) == 1;
    ok = ok && (a.empty() || std::fwrite(a.data(), 1, a.size(), f) == a.size());
    ok = ok && (b.empty() || std::fwrite(b.data(), 1, b.size(), f) == b.size());
    ok = (std::fclose(f) == 0) && ok;
    return ok ? SY_OK : fail(SY_ERR_IO, "write to %s failed", path);
}

sy_status sy_checkpoint_load(sy_queue_t qh, const char* path, const sy_stencil_params* p, void* u_prev, void* u_cur,
                             int64_t* step) {
    clear_error();
    Queue* q = nullptr;
    SY_TRY(check_queue(qh, &q));
    SY_TRY(stencil_param_checks(p));
    if (!path || !u_prev || !u_cur || !step) return fail(SY_ERR_NULL_POINTER, "NULL argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(SY_ERR_IO, "cannot open %s", path);
    Header h;
    if (std::fread(&h, sizeof h, 1, f) != 1 || h.magic != kMagic) {
        std::fclose(f);
        return fail(SY_ERR_IO, "%s is not a saved sy checkpoint", path);
    }
    if (h.dtype != p->dtype || h.ny != p->ny || h.nx != p->nx || h.radius != p->radius || h.c2 != p->c2) {
        std::fclose(f);
        return fail(SY_ERR_INVALID_ARGUMENT,
                    "%s holds a %lld x %lld grid (dtype %d, radius %d, c2 %g), not the one described", path,
                    (long long)h.ny, (long long)h.nx, h.dtype, h.radius, static_cast<double>(h.c2));
    }
    const size_t es = dtype_size(p->dtype), row = static_cast<size_t>(p->nx) * es;
    std::vector<unsigned char> a(row * static_cast<size_t>(p->ny)), b(a.size());
    bool ok = a.empty() || (std::fread(a.data(), 1, a.size(), f) == a.size() &&
                            std::fread(b.data(), 1, b.size(), f) == b.size());
    std::fclose(f);
    if (!ok) return fail(SY_ERR_IO, "%s is truncated", path);
    SY_TRY(use_device(q));
    if (!a.empty()) {
        const size_t dpitch = static_cast<size_t>(p->pitch) * es;
        SY_CUDA(cudaMemcpy2DAsync(u_prev, dpitch, a.data(), row, row, static_cast<size_t>(p->ny),
                                  cudaMemcpyHostToDevice, q->stream));
        SY_CUDA(cudaMemcpy2DAsync(u_cur, dpitch, b.data(), row, row, static_cast<size_t>(p->ny),
                                  cudaMemcpyHostToDevice, q->stream));
        SY_CUDA(cudaStreamSynchronize(q->stream));  // the host buffers die with this call
    }
    *step = h.step;
    return SY_OK;
}

}  // extern "C"
