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
#include <map>
#include <numeric>
#include <thread>
#include <tuple>
#include <vector>

#include "common.cuh"

using namespace iim;

namespace {
iim_opts opts_or_default(const iim_opts* o) {
    return o ? *o : iim_opts{IIM_FP64, 1e-10, 2000, 64, 12, 0, 0.0, 0};
}

// Lockstep groups of a batched call: the problems that can take the lockstep path (see
// lockstep.cu), bucketed by grid size and transform settings, largest grids first, each bucket
// split into groups of at most iim_set_lockstep's size (as even as possible; the groups run
// concurrently on their own streams); groups of one problem stay on the per-problem path.
std::vector<std::vector<int>> lockstep_groups(int n, iim_geometry const* geoms, const std::vector<int>& order,
                                              const iim_opts& o) {
    std::map<std::tuple<long, int, int, int, int, int>, std::vector<int>> b;
    for (int k : order) {
        iim_geometry g = geoms[k];
        if (lockstep_eligible(g, o))
            b[{-(long)g->nx * g->ny, g->nx, g->ny, g->wide_lines, g->cols_c, g->col_solver}].push_back(k);
    }
    std::vector<std::vector<int>> out;
    const int gmax = std::max(lockstep_group_size(), 1);
    for (auto& kv : b) {
        const std::vector<int>& v = kv.second;
        const int m = (int)v.size(), ng = (m + gmax - 1) / gmax;
        for (int gi = 0; gi < ng; ++gi) {
            std::vector<int> grp;
            for (int q = gi; q < m; q += ng) grp.push_back(v[q]);   // round robin: sizes differ by <= 1
            if (grp.size() >= 2) out.push_back(grp);
        }
    }
    (void)n;
    return out;
}

// Runs the lockstep groups, each on its own stream forked from `start`; `done[i]` is recorded
// on group i's stream.  While the per-kernel profiler is on, groups run host-driven one after
// the other on the calling thread.
struct LockstepRun {
    std::vector<std::vector<int>> groups;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    std::vector<void*> handles;
    bool host = false;
    ~LockstepRun() {
        for (cudaEvent_t e : done)
            if (e) cudaEventDestroy(e);
        for (cudaStream_t s : streams)
            if (s) cudaStreamDestroy(s);
    }
    iim_status open(cudaEvent_t start) {
        streams.assign(groups.size(), nullptr);
        done.assign(groups.size(), nullptr);
        handles.assign(groups.size(), nullptr);
        for (size_t i = 0; i < groups.size(); ++i) {
            IIM_TRY(cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking));
            IIM_TRY(cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming));
            IIM_TRY(cudaStreamWaitEvent(streams[i], start, 0));
        }
        return IIM_OK;
    }
    // after every stream of the call has been synchronised
    void finish(const iim_opts& o, std::vector<iim_status>& status, std::vector<iim_stats>& stats) {
        for (size_t i = 0; i < groups.size(); ++i)
            if (handles[i]) lockstep_finish(handles[i], groups[i], o, host, status, stats);
    }
};
}  // namespace

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
    // lockstep groups: one launch per step for all problems of a size bucket
    const iim_opts o = opts_or_default(opts);
    LockstepRun ls;
    ls.groups = lockstep_groups(n, geoms, order, o);
    ls.host = profiling_active();
    if (setup_st == IIM_OK) setup_st = ls.open(start);
    for (size_t i = 0; i < ls.groups.size() && setup_st == IIM_OK; ++i) {
        const iim_status e = lockstep_enqueue(ls.groups[i], geoms, omega, psi_b, psi_box, gamma, psibar, psi_out,
                                              ux_out, uy_out, o, ls.streams[i], ls.host, &ls.handles[i]);
        for (int k : ls.groups[i]) {
            enq[k] = 2;   // taken by the group
            if (e != IIM_OK) status[k] = e;
        }
        cudaEventRecord(ls.done[i], ls.streams[i]);
    }
    // whole-solve graphs: launched from here without waiting
    for (int q = 0; q < n && setup_st == IIM_OK; ++q) {
        const int k = order[q];
        if (enq[k] == 2) continue;
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
        for (size_t i = 0; i < ls.groups.size(); ++i) {
            cudaStreamSynchronize(ls.streams[i]);
            cudaStreamWaitEvent(cs, ls.done[i], 0);
        }
        for (int k = 0; k < n; ++k)
            if (enq[k] == 1) status[k] = solve_finish(geoms[k], opts, &stb[k]);
        ls.finish(o, status, stb);
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

// ---- the same on host buffers: each problem's inputs are copied in, solved and its outputs
// copied back on the problem's stream, so the copies of some problems overlap the solves of
// others.  Device staging arrays live in the geometry (allocated on first use).
namespace {
struct IoView {
    double *omega, *psi_b, *ring, *gamma, *psibar, *psi, *ux, *uy;
};
iim_status io_view(iim_geometry g, IoView* v) {
    const size_t nxy = (size_t)g->NX * g->NY, ncp = (size_t)std::max(g->ncp, 1), nring = 2 * (size_t)(g->nx + g->ny),
                 nb = (size_t)std::max(g->nb, 1);
    if (!g->io) IIM_TRY(cudaMalloc(&g->io, sizeof(double) * (4 * nxy + ncp + nring + 2 * nb)));
    double* p = g->io;
    v->omega = p; p += nxy;
    v->psi = p; p += nxy;
    v->ux = p; p += nxy;
    v->uy = p; p += nxy;
    v->psi_b = p; p += ncp;
    v->ring = p; p += nring;
    v->gamma = p; p += nb;
    v->psibar = p;
    return IIM_OK;
}
}  // namespace

// p lies in page-locked host memory that kernels can write through the same address
static bool device_writable_host(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost && a.devicePointer == p;
}

extern "C" iim_status iim_poisson_solve_batched_host(int n, iim_geometry const* geoms, const double* const* omega,
                                                     const double* const* psi_b, const double* const* psi_box,
                                                     const double* const* gamma, double* const* psibar,
                                                     double* const* psi_out, double* const* ux_out,
                                                     double* const* uy_out, const iim_opts* opts, iim_stats* stats,
                                                     int n_streams, iim_stream stream) {
    if (n < 0 || (n > 0 && (!geoms || !omega || !psi_out || !psibar || !psi_b))) return IIM_ERR_INVALID_ARG;
    if (n == 0) return IIM_OK;
    if (n_streams < 1) n_streams = 1;
    n_streams = std::min(n_streams, std::min(n, 64));
    for (int k = 0; k < n; ++k)
        if (!geoms[k]) return IIM_ERR_INVALID_ARG;
    for (int k = 0; k < n; ++k)
        for (int l = k + 1; l < n; ++l)
            if (geoms[k] == geoms[l]) return IIM_ERR_INVALID_ARG;
    std::vector<IoView> io(n);
    for (int k = 0; k < n; ++k) IIM_CHECK(io_view(geoms[k], &io[k]));
    // Outputs in page-locked host memory that the device can address (mapped under unified
    // addressing) are written there by the solve's last kernel; others are staged and copied.
    std::vector<char> direct(n, 0);
    for (int k = 0; k < n; ++k)
        direct[k] = device_writable_host(psi_out[k]) && (!ux_out || !ux_out[k] || device_writable_host(ux_out[k])) &&
                    (!uy_out || !uy_out[k] || device_writable_host(uy_out[k]));
    int dev = 0;
    IIM_TRY(cudaGetDevice(&dev));
    cudaStream_t cs = (cudaStream_t)stream;
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
    auto copy_in = [&](int k, cudaStream_t s) -> iim_status {
        iim_geometry g = geoms[k];
        const size_t nxy = (size_t)g->NX * g->NY;
        IIM_TRY(cudaMemcpyAsync(io[k].omega, omega[k], sizeof(double) * nxy, cudaMemcpyHostToDevice, s));
        if (g->ncp > 0)
            IIM_TRY(cudaMemcpyAsync(io[k].psi_b, psi_b[k], sizeof(double) * g->ncp, cudaMemcpyHostToDevice, s));
        if (psi_box && psi_box[k])
            IIM_TRY(cudaMemcpyAsync(io[k].ring, psi_box[k], sizeof(double) * 2 * (g->nx + g->ny),
                                    cudaMemcpyHostToDevice, s));
        if (gamma && gamma[k] && g->nb > 0)
            IIM_TRY(cudaMemcpyAsync(io[k].gamma, gamma[k], sizeof(double) * g->nb, cudaMemcpyHostToDevice, s));
        if (g->nb > 0)
            IIM_TRY(cudaMemcpyAsync(io[k].psibar, psibar[k], sizeof(double) * g->nb, cudaMemcpyHostToDevice, s));
        return IIM_OK;
    };
    auto copy_out = [&](int k, cudaStream_t s) -> iim_status {
        iim_geometry g = geoms[k];
        const size_t nxy = (size_t)g->NX * g->NY;
        if (!direct[k]) {
            IIM_TRY(cudaMemcpyAsync(psi_out[k], io[k].psi, sizeof(double) * nxy, cudaMemcpyDeviceToHost, s));
            if (ux_out && ux_out[k])
                IIM_TRY(cudaMemcpyAsync(ux_out[k], io[k].ux, sizeof(double) * nxy, cudaMemcpyDeviceToHost, s));
            if (uy_out && uy_out[k])
                IIM_TRY(cudaMemcpyAsync(uy_out[k], io[k].uy, sizeof(double) * nxy, cudaMemcpyDeviceToHost, s));
        }
        if (g->nb > 0)
            IIM_TRY(cudaMemcpyAsync(psibar[k], io[k].psibar, sizeof(double) * g->nb, cudaMemcpyDeviceToHost, s));
        return IIM_OK;
    };
    auto dev_args = [&](int k, const double** ring, const double** gam, double** psi, double** ux, double** uy) {
        *ring = (psi_box && psi_box[k]) ? io[k].ring : nullptr;
        *gam = (gamma && gamma[k]) ? io[k].gamma : nullptr;
        *psi = direct[k] ? psi_out[k] : io[k].psi;
        *ux = (ux_out && ux_out[k]) ? (direct[k] ? ux_out[k] : io[k].ux) : nullptr;
        *uy = (uy_out && uy_out[k]) ? (direct[k] ? uy_out[k] : io[k].uy) : nullptr;
    };
    std::vector<iim_status> status(n, IIM_OK);
    std::vector<int> enq(n, -1);
    std::vector<iim_stats> stb(n);
    // lockstep groups: inputs copied in on the group's stream, one lockstep solve, outputs out
    const iim_opts o = opts_or_default(opts);
    LockstepRun ls;
    ls.groups = lockstep_groups(n, geoms, order, o);
    ls.host = profiling_active();
    if (setup_st == IIM_OK) setup_st = ls.open(start);
    if (!ls.groups.empty() && setup_st == IIM_OK) {
        std::vector<const double*> d_om(n), d_pb(n), d_ring(n), d_gam(n);
        std::vector<double*> d_pbar(n), d_psi(n), d_ux(n), d_uy(n);
        for (int k = 0; k < n; ++k) {
            dev_args(k, &d_ring[k], &d_gam[k], &d_psi[k], &d_ux[k], &d_uy[k]);
            d_om[k] = io[k].omega;
            d_pb[k] = io[k].psi_b;
            d_pbar[k] = io[k].psibar;
        }
        for (size_t i = 0; i < ls.groups.size(); ++i) {
            cudaStream_t s = ls.streams[i];
            iim_status e = IIM_OK;
            for (int k : ls.groups[i])
                if (e == IIM_OK) e = copy_in(k, s);
            if (e == IIM_OK)
                e = lockstep_enqueue(ls.groups[i], geoms, d_om.data(), d_pb.data(), d_ring.data(), d_gam.data(),
                                     d_pbar.data(), d_psi.data(), d_ux.data(), d_uy.data(), o, s, ls.host,
                                     &ls.handles[i]);
            for (int k : ls.groups[i])
                if (e == IIM_OK) e = copy_out(k, s);
            for (int k : ls.groups[i]) {
                enq[k] = 2;
                if (e != IIM_OK) status[k] = e;
            }
            cudaEventRecord(ls.done[i], s);
        }
    }
    for (int q = 0; q < n && setup_st == IIM_OK; ++q) {
        const int k = order[q];
        if (enq[k] == 2) continue;
        cudaStream_t s = ws[q % n_streams];
        int e = -1;
        const double* ring;
        const double* gam;
        double *psi, *ux, *uy;
        dev_args(k, &ring, &gam, &psi, &ux, &uy);
        // the graph path applies after a first solve on the geometry: ask before copying
        iim_geometry g = geoms[k];
        const bool graph_ready = g->host_solves > 0 && !g->solve_graph_failed;
        if (!graph_ready) continue;
        status[k] = copy_in(k, s);
        if (status[k] == IIM_OK)
            status[k] = solve_enqueue(g, io[k].omega, io[k].psi_b, ring, gam, io[k].psibar, psi, ux, uy, opts, &stb[k],
                                      s, &e);
        if (status[k] == IIM_OK && e >= 0) status[k] = copy_out(k, s);
        enq[k] = status[k] == IIM_OK ? e : 0;
        if (enq[k] < 0) enq[k] = -2;   // copied in but not solved: solved by a worker below
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
            const double* ring;
            const double* gam;
            double *psi, *ux, *uy;
            dev_args(k, &ring, &gam, &psi, &ux, &uy);
            iim_status st = enq[k] == -2 ? IIM_OK : copy_in(k, ws[t]);
            iim_stats sk;
            if (st == IIM_OK)
                st = iim_poisson_solve(geoms[k], io[k].omega, io[k].psi_b, ring, gam, io[k].psibar, psi, ux, uy,
                                       nullptr, opts, &sk, (iim_stream)ws[t]);
            if (st == IIM_OK) st = copy_out(k, ws[t]);
            status[k] = st;
            stb[k] = sk;
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
        for (size_t i = 0; i < ls.groups.size(); ++i) {
            cudaStreamSynchronize(ls.streams[i]);
            cudaStreamWaitEvent(cs, ls.done[i], 0);
        }
        for (int k = 0; k < n; ++k)
            if (enq[k] == 1) status[k] = solve_finish(geoms[k], opts, &stb[k]);
        ls.finish(o, status, stb);
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
