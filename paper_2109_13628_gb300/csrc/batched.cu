// Batched IIM Poisson solves: many independent problems (each with its own geometry, grid
// size and right-hand side) in flight at once, on n_streams non-blocking streams, largest
// problems first (longest-processing-time order).  Problems whose geometry has its whole-solve
// graph (every solve after the first on a geometry) are launched from this thread, one graph
// launch each and no wait in between; the rest (first solves: host-driven, with their
// set-up) are taken by a pool of worker threads, one per stream.  The GPU overlaps the
// latency-bound kernels of different problems.  The caller's stream is joined in both
// directions with events, so the call is stream-ordered for the caller.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>
#include <thread>
#include <vector>

#include "common.cuh"

using namespace iim;

extern "C" iim_status iim_poisson_solve_batched(int n, iim_geometry const* geoms, const double* const* omega,
                                                const double* const* psi_b, const double* const* psi_box,
                                                const double* const* gamma, double* const* psibar,
                                                double* const* psi_out, double* const* ux_out, double* const* uy_out,
                                                const iim_opts* opts, iim_stats* stats, int n_streams,
                                                iim_stream stream) {
    if (n < 0 || (n > 0 && (!geoms || !omega || !psi_out || !psibar || !psi_b))) return IIM_ERR_INVALID_ARG;
    if (n == 0) return IIM_OK;
    if (n_streams < 1) n_streams = 1;
    n_streams = std::min(n_streams, std::min(n, 64));
    for (int k = 0; k < n; ++k)
        if (!geoms[k]) return IIM_ERR_INVALID_ARG;
    for (int k = 0; k < n; ++k)
        for (int l = k + 1; l < n; ++l)
            if (geoms[k] == geoms[l]) return IIM_ERR_INVALID_ARG;   // problems must not share a workspace
    int dev = 0;
    IIM_TRY(cudaGetDevice(&dev));
    cudaStream_t cs = (cudaStream_t)stream;
    // order: largest problems first
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (long)geoms[a]->nx * geoms[a]->ny > (long)geoms[b]->nx * geoms[b]->ny;
    });
    cudaEvent_t start = nullptr;
    IIM_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    IIM_TRY(cudaEventRecord(start, cs));
    std::vector<cudaStream_t> ws(n_streams, nullptr);
    std::vector<cudaEvent_t> done(n_streams, nullptr);
    iim_status setup_st = IIM_OK;
    for (int t = 0; t < n_streams && setup_st == IIM_OK; ++t) {
        if (cudaStreamCreateWithFlags(&ws[t], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&done[t], cudaEventDisableTiming) != cudaSuccess ||
            cudaStreamWaitEvent(ws[t], start, 0) != cudaSuccess)
            setup_st = IIM_ERR_CUDA;
    }
    std::vector<iim_status> status(n, IIM_OK);
    std::vector<int> enq(n, -1);
    std::vector<iim_stats> stb(n);
    // whole-solve graphs: launched from here without waiting
    for (int q = 0; q < n && setup_st == IIM_OK; ++q) {
        const int k = order[q];
        status[k] = solve_enqueue(geoms[k], omega[k], psi_b[k], psi_box ? psi_box[k] : nullptr,
                                  gamma ? gamma[k] : nullptr, psibar[k], psi_out[k], ux_out ? ux_out[k] : nullptr,
                                  uy_out ? uy_out[k] : nullptr, opts, &stb[k], ws[q % n_streams], &enq[k]);
        if (status[k] != IIM_OK) enq[k] = 0;
    }
    std::vector<int> rest;
    for (int q = 0; q < n; ++q)
        if (enq[order[q]] < 0) rest.push_back(order[q]);
    std::atomic<int> next{0};
    auto worker = [&](int t) {
        cudaSetDevice(dev);
        for (;;) {
            const int q = next.fetch_add(1);
            if (q >= (int)rest.size()) break;
            const int k = rest[q];
            iim_stats st;
            status[k] = iim_poisson_solve(geoms[k], omega[k], psi_b[k], psi_box ? psi_box[k] : nullptr,
                                          gamma ? gamma[k] : nullptr, psibar[k], psi_out[k],
                                          ux_out ? ux_out[k] : nullptr, uy_out ? uy_out[k] : nullptr, nullptr, opts,
                                          &st, (iim_stream)ws[t]);
            stb[k] = st;
        }
        cudaEventRecord(done[t], ws[t]);
    };
    if (setup_st == IIM_OK) {
        std::vector<std::thread> pool;
        const int nthreads = rest.empty() ? 1 : n_streams;
        for (int t = 1; t < nthreads; ++t) pool.emplace_back(worker, t);
        worker(0);
        for (auto& th : pool) th.join();
        for (int t = 1; t < n_streams; ++t)
            if (t >= nthreads) cudaEventRecord(done[t], ws[t]);
        for (int t = 0; t < n_streams; ++t) {
            cudaStreamSynchronize(ws[t]);
            cudaStreamWaitEvent(cs, done[t], 0);
        }
        for (int k = 0; k < n; ++k)
            if (enq[k] == 1) status[k] = solve_finish(geoms[k], opts, &stb[k]);
        if (stats)
            for (int k = 0; k < n; ++k) stats[k] = stb[k];
    }
    for (int t = 0; t < n_streams; ++t) {
        if (done[t]) cudaEventDestroy(done[t]);
        if (ws[t]) cudaStreamDestroy(ws[t]);
    }
    cudaEventDestroy(start);
    if (setup_st != IIM_OK) return setup_st;
    for (int k = 0; k < n; ++k)
        if (status[k] != IIM_OK) return status[k];
    return IIM_OK;
}
