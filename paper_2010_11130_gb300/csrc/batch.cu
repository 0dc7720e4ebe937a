// Independent problems at once: one host thread and one stream per problem.
//
// The first pass of every level runs on a single warp, so one setup occupies
// one SM at a time for most of its duration; independent systems (several
// space-time problems, or the forward and adjoint systems) set up on separate
// streams run side by side on the GPU's other SMs.  Every call below is the
// single-problem entry point run on its own host thread; library allocations
// inside a call are stream-ordered (air_dmalloc), so no call synchronises the
// device and the streams overlap.
#include <thread>
#include <vector>

#include "air_internal.cuh"

namespace {

template <typename F>
int run_all(int count, void *const *streams, int *status, F &&call) {
    int dev = 0;
    AIR_CUDA(cudaGetDevice(&dev));
    std::vector<cudaStream_t> own((size_t)count, nullptr);
    std::vector<int> st((size_t)count, AIR_OK);
    for (int k = 0; k < count; ++k) {
        if (streams && streams[k]) continue;
        if (cudaStreamCreateWithFlags(&own[(size_t)k], cudaStreamNonBlocking) != cudaSuccess) {
            for (int q = 0; q < k; ++q)
                if (own[(size_t)q]) cudaStreamDestroy(own[(size_t)q]);
            return AIR_ERR_CUDA;
        }
    }
    auto stream_of = [&](int k) { return (streams && streams[k]) ? (cudaStream_t)streams[k] : own[(size_t)k]; };
    std::vector<std::thread> th;
    th.reserve((size_t)count);
    for (int k = 0; k < count; ++k) {
        try {
            th.emplace_back([&, k] {
                cudaSetDevice(dev);
                st[(size_t)k] = call(k, stream_of(k));
            });
        } catch (...) {
            st[(size_t)k] = call(k, stream_of(k));   // no thread available: run it here
        }
    }
    for (auto &t : th) t.join();
    for (int k = 0; k < count; ++k) {
        if (own[(size_t)k]) {
            cudaStreamSynchronize(own[(size_t)k]);
            cudaStreamDestroy(own[(size_t)k]);
        }
    }
    int first = AIR_OK;
    for (int k = 0; k < count; ++k) {
        if (status) status[k] = st[(size_t)k];
        if (first == AIR_OK && st[(size_t)k] < 0) first = st[(size_t)k];
    }
    return first;
}

}  // namespace

extern "C" int air_setup_batch(int count, const air_csr *A, double theta, int distance, const air_options *opt,
                               void *const *streams, air_hierarchy **out, int *status) {
    if (count < 0 || (count > 0 && (!A || !out))) return AIR_ERR_INVALID_ARG;
    for (int k = 0; k < count; ++k) out[k] = nullptr;
    return run_all(count, streams, status, [&](int k, cudaStream_t s) {
        return air_setup(&A[k], theta, distance, opt, (void *)s, &out[k]);
    });
}

extern "C" int air_gmres_solve_batch(int count, const air_csr *A, const air_hierarchy *const *H,
                                     const double *const *b, double *const *x, double rtol, void *const *streams,
                                     air_solve_info *info, int *status) {
    if (count < 0 || (count > 0 && (!A || !H || !b || !x))) return AIR_ERR_INVALID_ARG;
    for (int k = 0; k < count; ++k)
        for (int q = 0; q < k; ++q)
            if (H[k] == H[q]) return AIR_ERR_INVALID_ARG;   // a hierarchy's workspace serves one solve at a time
    return run_all(count, streams, status, [&](int k, cudaStream_t s) {
        return air_gmres_solve(&A[k], H[k], b[k], x[k], rtol, (void *)s, info ? &info[k] : nullptr);
    });
}
