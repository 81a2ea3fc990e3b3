// GMM objective and gradient from host memory (gmm_vjp_host): the points stream
// to the device in chunks through two staging buffers, the copy of chunk c + 1
// (on a library stream) overlapping the reverse pass on chunk c (on the
// caller's stream); the chunks' Accum sums add up in one exchange vector (the
// associativity of Accum, Sec. 2.3.2), which is finished once for all points;
// the gradient and the objective go back to host memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "common.cuh"
#include "gmm_internal.cuh"
#include "trace.cuh"

namespace gpa {
namespace {

size_t h256(size_t v) { return (v + 255) & ~(size_t)255; }

// chunk size: a multiple of 128 points, at least 128, at most n rounded up
int64_t host_chunk(int64_t n, int64_t chunk_points) {
    int64_t c = chunk_points <= 0 ? ((int64_t)1 << 19) : chunk_points;
    c = (c / 128) * 128;
    if (c < 128) c = 128;
    const int64_t nr = (n + 127) / 128 * 128;
    return c < nr ? c : nr;
}

struct HostLayout {
    size_t off_alpha, off_mu, off_q, off_l, off_galpha, off_gmu, off_gq, off_gl, off_out, off_exch, off_stage[2],
        off_ws, ws_bytes, total;
};

HostLayout host_layout(int64_t n, int d, int k, int prec, int64_t chunk) {
    HostLayout H{};
    const size_t t = (size_t)d * (d - 1) / 2;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = h256(off + (bytes ? bytes : 1));
        return o;
    };
    H.off_alpha = take(4 * (size_t)k);
    H.off_mu = take(4 * (size_t)k * d);
    H.off_q = take(4 * (size_t)k * d);
    H.off_l = take(4 * (size_t)k * t);
    H.off_galpha = take(4 * (size_t)k);
    H.off_gmu = take(4 * (size_t)k * d);
    H.off_gq = take(4 * (size_t)k * d);
    H.off_gl = take(4 * (size_t)k * t);
    H.off_out = take(8);
    H.off_exch = take(8 * (size_t)gmm_exchange_len(d, k));
    H.off_stage[0] = take(4 * (size_t)chunk * d);
    H.off_stage[1] = take(4 * (size_t)chunk * d);
    H.ws_bytes = gpa_gmm_workspace_bytes(chunk, d, k, prec, 0);
    H.off_ws = take(H.ws_bytes);
    H.total = off;
    (void)n;
    return H;
}

// The library's copy stream, one per device, made on first use and kept for
// the process.
constexpr int kHostMaxDevices = 64;
cudaStream_t g_copy_stream[kHostMaxDevices];
std::mutex g_copy_mu;

cudaStream_t copy_stream() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kHostMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_copy_mu);
    if (!g_copy_stream[dev] && cudaStreamCreateWithFlags(&g_copy_stream[dev], cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        g_copy_stream[dev] = nullptr;
    }
    return g_copy_stream[dev];
}

}  // namespace
}  // namespace gpa

using namespace gpa;

extern "C" size_t gpa_gmm_vjp_host_workspace_bytes(int64_t n, int32_t d, int32_t k, int32_t prec,
                                                   int64_t chunk_points) {
    if (n < 1 || d < 1 || d > 128 || k < 1 || k > 4096) return 0;
    if (prec != GPA_PREC_FP32 && prec != GPA_PREC_BF16_TC) return 0;
    const HostLayout H = host_layout(n, d, k, prec, host_chunk(n, chunk_points));
    return H.ws_bytes ? H.total : 0;
}

extern "C" int gmm_vjp_host(const float* x, const float* alpha, const float* mu, const float* q, const float* l,
                            int64_t n, int32_t d, int32_t k, double gamma, int32_t m, int32_t prec, double seed,
                            float* d_alpha, float* d_mu, float* d_q, float* d_l, double* out,
                            int64_t chunk_points, void* ws, size_t ws_bytes, int32_t* dev_status,
                            gpa_stream_t stream) {
    if (!x || !alpha || !mu || !q || (d > 1 && !l) || !d_alpha || !d_mu || !d_q || (d > 1 && !d_l) || !ws)
        return GPA_ERR_ARG;
    if (n < 1 || d < 1 || d > 128 || k < 1 || k > 4096 || !(gamma > 0.0)) return GPA_ERR_ARG;
    if (prec != GPA_PREC_FP32 && prec != GPA_PREC_BF16_TC) return GPA_ERR_ARG;
    if (prec == GPA_PREC_BF16_TC && !gmm_tc_supported(d)) return GPA_ERR_UNSUPPORTED;
    if (((uintptr_t)ws) & 255) return GPA_ERR_ALIGN;
    const int64_t chunk = host_chunk(n, chunk_points);
    const HostLayout H = host_layout(n, d, k, prec, chunk);
    if (H.ws_bytes == 0 || ws_bytes < H.total) return GPA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream, cs = copy_stream();
    if (!cs) return GPA_ERR_CUDA;
    char* w = (char*)ws;
    const size_t t = (size_t)d * (d - 1) / 2;
    float *a_d = (float*)(w + H.off_alpha), *mu_d = (float*)(w + H.off_mu), *q_d = (float*)(w + H.off_q),
          *l_d = (float*)(w + H.off_l);
    float *ga = (float*)(w + H.off_galpha), *gm = (float*)(w + H.off_gmu), *gq = (float*)(w + H.off_gq),
          *gl = (float*)(w + H.off_gl);
    double* out_d = (double*)(w + H.off_out);
    double* exch = (double*)(w + H.off_exch);
    const int64_t elen = gmm_exchange_len(d, k);
    // parameters in, accumulators cleared (all on the caller's stream)
    bool ok = cudaMemcpyAsync(a_d, alpha, 4 * (size_t)k, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(mu_d, mu, 4 * (size_t)k * d, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(q_d, q, 4 * (size_t)k * d, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              (t == 0 || cudaMemcpyAsync(l_d, l, 4 * (size_t)k * t, cudaMemcpyHostToDevice, s) == cudaSuccess) &&
              cudaMemsetAsync(w + H.off_galpha, 0, H.off_out - H.off_galpha, s) == cudaSuccess &&
              cudaMemsetAsync(exch, 0, 8 * (size_t)elen, s) == cudaSuccess;
    if (!ok) return GPA_ERR_CUDA;
    // events: the staging buffers' copies done (copied) and their readers done (freed)
    // (fork / join: the copy stream starts after, and is joined back into, the caller's stream)
    cudaEvent_t ev[6];  // fork, join, copied[2], freed[2]
    int made = 0;
    while (made < 6 && cudaEventCreateWithFlags(&ev[made], cudaEventDisableTiming) == cudaSuccess) ++made;
    cudaEvent_t fork = ev[0], join = ev[1], copied[2] = {ev[2], ev[3]}, freed[2] = {ev[4], ev[5]};
    int rc = made == 6 ? GPA_OK : GPA_ERR_CUDA;
    // the copy stream starts after the work already on the caller's stream
    // (which may still read the staging buffers)
    if (!rc && (cudaEventRecord(fork, s) != cudaSuccess || cudaStreamWaitEvent(cs, fork, 0) != cudaSuccess))
        rc = GPA_ERR_CUDA;
    // the first chunk is a quarter of the others: its copy is the one that
    // nothing overlaps
    const int64_t first = (chunk / 4) / 128 * 128 >= 128 ? (chunk / 4) / 128 * 128 : 128;
    int64_t b0 = 0;
    for (int c = 0; !rc && b0 < n; ++c) {
        const int64_t len = (c == 0 ? (first < n ? first : n) : (chunk < n - b0 ? chunk : n - b0));
        const int slot = c & 1;
        float* stage = (float*)(w + H.off_stage[slot]);
        if (c >= 2 && cudaStreamWaitEvent(cs, freed[slot], 0) != cudaSuccess) rc = GPA_ERR_CUDA;
        if (!rc && (cudaMemcpyAsync(stage, x + b0 * d, 4 * (size_t)len * d, cudaMemcpyHostToDevice, cs) !=
                        cudaSuccess ||
                    cudaEventRecord(copied[slot], cs) != cudaSuccess || cudaStreamWaitEvent(s, copied[slot], 0) !=
                                                                            cudaSuccess))
            rc = GPA_ERR_CUDA;
        if (!rc)
            rc = gmm_vjp_partial(stage, a_d, mu_d, q_d, l_d, len, d, k, gamma, m, prec, nullptr, nullptr, seed, exch,
                                 w + H.off_ws, H.ws_bytes, dev_status, stream);
        if (!rc && cudaEventRecord(freed[slot], s) != cudaSuccess) rc = GPA_ERR_CUDA;
        b0 += len;
    }
    // every copy is ordered before what follows on the caller's stream, also
    // when the loop above stopped early
    if (made == 6 && (cudaEventRecord(join, cs) != cudaSuccess || cudaStreamWaitEvent(s, join, 0) != cudaSuccess))
        rc = GPA_ERR_CUDA;
    if (!rc)
        rc = gmm_vjp_finalize(a_d, mu_d, q_d, l_d, n, d, k, gamma, m, prec, seed, exch, ga, gm, gq, t ? gl : nullptr,
                              out_d, w + H.off_ws, H.ws_bytes, dev_status, stream);
    // results out (written, not added: the host buffers are outputs only)
    if (!rc && (cudaMemcpyAsync(d_alpha, ga, 4 * (size_t)k, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaMemcpyAsync(d_mu, gm, 4 * (size_t)k * d, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaMemcpyAsync(d_q, gq, 4 * (size_t)k * d, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                (t && cudaMemcpyAsync(d_l, gl, 4 * (size_t)k * t, cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
                (out && cudaMemcpyAsync(out, out_d, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)))
        rc = GPA_ERR_CUDA;
    for (int e = 0; e < made; ++e) cudaEventDestroy(ev[e]);  // released once their work completes
    if (rc == GPA_ERR_CUDA) (void)cudaGetLastError();
    return rc;
}
