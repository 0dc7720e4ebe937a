// Independent problems at once.
//
// Setup runs the problems level by level in lockstep: each problem's
// strength, transpose and C/F splitting of level l run on its own host thread
// and stream (the first pass of a level is one warp, so the problems' first
// passes run side by side on different SMs), then the local l-AIR solves of
// level l of every problem go out as one launch (air_lair_solve_batch: one
// index range over all problems' C points), then each problem builds its P
// and A_{l+1} on its own thread again.  The results are those of the
// single-problem setup bit for bit: every step is the same kernel on the same
// data, and a local solve's arithmetic does not depend on the launch it runs
// in.  Library allocations inside a call are stream-ordered (air_dmalloc), so
// the streams overlap.
//
// Solve runs the problems' flexible GMRES in lockstep rounds on one host
// thread, with the V-cycles of every problem in one CUDA graph (below).
#include <thread>
#include <vector>

#include "air_internal.cuh"

namespace {

// fn(k, stream of k) for every k with run[k], one host thread each (inline
// when only one runs), with k's stream as the thread's library call stream.
template <typename F>
void for_each_problem(int count, const std::vector<char> &run, const std::vector<cudaStream_t> &str, int dev,
                      std::vector<int> &st, F &&fn) {
    auto one = [&](int k) {
        cudaSetDevice(dev);
        AirCallStream call(str[(size_t)k]);
        st[(size_t)k] = fn(k, str[(size_t)k]);
    };
    std::vector<int> ks;
    for (int k = 0; k < count; ++k)
        if (run[(size_t)k]) ks.push_back(k);
    if (ks.size() == 1) {
        one(ks[0]);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(ks.size());
    for (int k : ks) {
        try {
            th.emplace_back(one, k);
        } catch (...) {
            one(k);                                  // no thread available: run it here
        }
    }
    for (auto &t : th) t.join();
}

}  // namespace

extern "C" int air_setup_batch(int count, const air_csr *A, double theta, int distance, const air_options *opt,
                               void *const *streams, air_hierarchy **out, int *status) {
    if (count < 0 || (count > 0 && (!A || !out))) return AIR_ERR_INVALID_ARG;
    for (int k = 0; k < count; ++k) out[k] = nullptr;
    if (count == 0) return AIR_OK;
    air_options o;
    const int oc = air_check_options(theta, distance, opt, &o);
    if (oc != AIR_OK) {
        for (int k = 0; status && k < count; ++k) status[k] = oc;
        return oc;
    }
    int dev = 0;
    AIR_CUDA(cudaGetDevice(&dev));
    const size_t nk = (size_t)count;
    std::vector<int> st(nk, AIR_OK);
    std::vector<air_hierarchy *> H(nk, nullptr);
    std::vector<cudaStream_t> str(nk, nullptr), own(nk, nullptr);
    for (int k = 0; k < count; ++k) {
        const air_csr &a = A[k];
        if (!a.row_ptr || !a.col || !a.val || a.n_rows <= 0 || a.n_rows != a.n_cols || a.nnz < a.n_rows ||
            a.n_rows > INT32_MAX) {
            st[(size_t)k] = AIR_ERR_INVALID_ARG;
            continue;
        }
        H[(size_t)k] = new (std::nothrow) air_hierarchy();
        if (!H[(size_t)k]) {
            st[(size_t)k] = AIR_ERR_OOM;
            continue;
        }
        if (streams && streams[k]) {
            str[(size_t)k] = (cudaStream_t)streams[k];
        } else if (cudaStreamCreateWithFlags(&own[(size_t)k], cudaStreamNonBlocking) == cudaSuccess) {
            str[(size_t)k] = own[(size_t)k];
        } else {
            st[(size_t)k] = AIR_ERR_CUDA;
        }
    }
    auto ok = [&](int k) { return st[(size_t)k] == AIR_OK && H[(size_t)k] != nullptr; };
    std::vector<char> run(nk, 0);
    for (int k = 0; k < count; ++k) run[(size_t)k] = ok(k);
    for_each_problem(count, run, str, dev, st,
                     [&](int k, cudaStream_t s) { return air_setup_begin(&A[k], &o, s, H[(size_t)k]); });
    // level by level
    std::vector<char> building(nk, 0);
    for (int k = 0; k < count; ++k) building[(size_t)k] = ok(k);
    std::vector<AirCoarsen> C(nk);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    AIR_CUDA(cudaEventCreate(&ev[0]));
    AIR_CUDA(cudaEventCreate(&ev[1]));
    for (int l = 0;; ++l) {
        for (int k = 0; k < count; ++k) {
            if (!building[(size_t)k]) continue;
            H[(size_t)k]->nlev = l + 1;
            if (air_setup_is_coarsest(H[(size_t)k], l)) building[(size_t)k] = 0;
        }
        bool any = false;
        for (int k = 0; k < count; ++k) any = any || building[(size_t)k];
        if (!any) break;
        for_each_problem(count, building, str, dev, st, [&](int k, cudaStream_t s) {
            return air_coarsen_split(H[(size_t)k], l, s, &C[(size_t)k]);
        });
        std::vector<const AirLevel *> lv;
        std::vector<int32_t> mm;
        std::vector<int64_t *> ns;
        std::vector<int> jk;
        for (int k = 0; k < count; ++k) {
            if (!building[(size_t)k]) continue;
            if (!ok(k) || C[(size_t)k].stop) {
                building[(size_t)k] = 0;
                continue;
            }
            jk.push_back(k);
            lv.push_back(&C[(size_t)k].LS);
            mm.push_back(H[(size_t)k]->lev[l].max_m);
            ns.push_back(C[(size_t)k].dsing);
        }
        if (jk.empty()) break;
        // a4 for every problem at once
        cudaStream_t s0 = str[(size_t)jk[0]];
        int bst = AIR_OK;
        {
            AirCallStream call(s0);
            cudaEventRecord(ev[0], s0);
            bst = air_lair_solve_batch((int)jk.size(), lv.data(), mm.data(), o.distance, ns.data(), s0);
            cudaEventRecord(ev[1], s0);
        }
        float ms = 0.f;
        if (bst == AIR_OK && cudaEventSynchronize(ev[1]) == cudaSuccess &&
            cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess) {
            for (int k : jk) air_add_phase_ms(H[(size_t)k], 3, (double)ms);
        }
        if (bst != AIR_OK) {
            for (int k : jk) {
                st[(size_t)k] = bst;
                building[(size_t)k] = 0;
            }
            break;
        }
        for_each_problem(count, building, str, dev, st, [&](int k, cudaStream_t s) {
            return air_coarsen_finish(H[(size_t)k], l, s, &C[(size_t)k]);
        });
        for (int k = 0; k < count; ++k)
            if (!ok(k)) building[(size_t)k] = 0;
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    for (int k = 0; k < count; ++k) run[(size_t)k] = ok(k);
    for_each_problem(count, run, str, dev, st,
                     [&](int k, cudaStream_t s) { return air_setup_end(H[(size_t)k], s); });
    int first = AIR_OK;
    for (int k = 0; k < count; ++k) {
        if (str[(size_t)k]) cudaStreamSynchronize(str[(size_t)k]);
        if (st[(size_t)k] != AIR_OK) {
            if (H[(size_t)k]) air_free(H[(size_t)k]);
            H[(size_t)k] = nullptr;
        }
        out[k] = H[(size_t)k];
        if (status) status[k] = st[(size_t)k];
        if (first == AIR_OK && st[(size_t)k] != AIR_OK) first = st[(size_t)k];
        if (own[(size_t)k]) cudaStreamDestroy(own[(size_t)k]);
    }
    return first;
}

namespace {

// One CUDA graph for a set of hierarchies: a gather of the caller's vectors
// into every member's lev[0].b (job table d_in), the members' V-cycles as
// parallel branches, and a scatter of every lev[0].x back (job table d_out).
// Table entries of n = 0 are skipped, so one graph serves every step in which
// its members are the hierarchies still solving.
struct BatchVcycle {
    cudaGraphExec_t exec = nullptr;
    unsigned long long kernels = 0;
    std::vector<int> members;
    ~BatchVcycle() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

int build_batch_vcycle(const std::vector<air_hierarchy *> &H, const std::vector<int> &members, int count,
                       const AirConvJob *d_in, const AirConvJob *d_out, BatchVcycle *bv) {
    if (bv->exec) cudaGraphExecDestroy(bv->exec);
    bv->exec = nullptr;
    bv->members = members;
    cudaStream_t cs = nullptr;
    AIR_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    std::vector<cudaStream_t> br(members.size(), nullptr);
    std::vector<cudaEvent_t> ev(members.size() + 1, nullptr);
    int st = AIR_OK;
    for (auto &b : br)
        if (st == AIR_OK && cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking) != cudaSuccess) st = AIR_ERR_CUDA;
    for (auto &e : ev)
        if (st == AIR_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) st = AIR_ERR_CUDA;
    cudaGraph_t g = nullptr;
    const unsigned long long c0 = air_launch_counter_add(0);
    if (st == AIR_OK && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        int cst = air_convert_batch(count, d_in, cs);
        if (cst == AIR_OK && cudaEventRecord(ev[0], cs) != cudaSuccess) cst = AIR_ERR_CUDA;
        for (size_t q = 0; cst == AIR_OK && q < members.size(); ++q) {
            AirCallStream call(br[q]);
            if (cudaStreamWaitEvent(br[q], ev[0], 0) != cudaSuccess) cst = AIR_ERR_CUDA;
            if (cst == AIR_OK) cst = air_vcycle_staged(H[(size_t)members[q]], br[q]);
            if (cst == AIR_OK && cudaEventRecord(ev[q + 1], br[q]) != cudaSuccess) cst = AIR_ERR_CUDA;
            if (cst == AIR_OK && cudaStreamWaitEvent(cs, ev[q + 1], 0) != cudaSuccess) cst = AIR_ERR_CUDA;
        }
        if (cst == AIR_OK) cst = air_convert_batch(count, d_out, cs);
        const cudaError_t e = cudaStreamEndCapture(cs, &g);
        st = cst != AIR_OK ? cst : (e == cudaSuccess ? AIR_OK : AIR_ERR_CUDA);
    } else if (st == AIR_OK) {
        st = AIR_ERR_CUDA;
    }
    const unsigned long long c1 = air_launch_counter_add(0);
    air_launch_counter_sub(c1 - c0);   // captured, not yet run
    if (st == AIR_OK && cudaGraphInstantiate(&bv->exec, g, 0) != cudaSuccess) {
        bv->exec = nullptr;
        st = AIR_ERR_CUDA;
    }
    bv->kernels = c1 - c0;
    if (g) cudaGraphDestroy(g);
    for (auto e : ev)
        if (e) cudaEventDestroy(e);
    for (auto b : br)
        if (b) cudaStreamDestroy(b);
    cudaStreamDestroy(cs);
    if (st != AIR_OK) (void)cudaGetLastError();
    return st;
}

}  // namespace

// Lockstep flexible GMRES over independent problems.  Every host round, the
// problems in an Arnoldi step get their V-cycles from one graph launch
// (BatchVcycle, rebuilt only when a problem finishes), then each problem's
// own step (matrix product, CGS2, Givens) or cycle start runs on its stream;
// one synchronisation per round serves all problems.  Each problem runs the
// single-problem solve's phases (air_gmres_*) with the same kernels on the
// same data, so its result is that solve's bit for bit.
extern "C" int air_gmres_solve_batch(int count, const air_csr *A, const air_hierarchy *const *H,
                                     const double *const *b, double *const *x, double rtol, void *const *streams,
                                     air_solve_info *info, int *status) {
    if (count < 0 || (count > 0 && (!A || !H || !b || !x))) return AIR_ERR_INVALID_ARG;
    for (int k = 0; k < count; ++k)
        for (int q = 0; q < k; ++q)
            if (H[k] == H[q]) return AIR_ERR_INVALID_ARG;   // a hierarchy's workspace serves one solve at a time
    if (count == 0) return AIR_OK;
    const size_t nk = (size_t)count;
    std::vector<int> st(nk, AIR_OK);
    std::vector<air_hierarchy *> Hm(nk, nullptr);
    std::vector<cudaStream_t> str(nk, nullptr), own(nk, nullptr);
    std::vector<AirGmres> g(nk);
    std::vector<air_solve_info> local(nk);
    std::vector<const double *> bd(nk, nullptr);
    std::vector<double *> xd(nk, nullptr);
    cudaStream_t ms = nullptr;
    AIR_CUDA(cudaStreamCreateWithFlags(&ms, cudaStreamNonBlocking));
    AirConvJob *h_tab = nullptr, *d_tab = nullptr;
    std::vector<cudaEvent_t> ev(nk + 1, nullptr);
    int first = AIR_OK;
    auto fail = [&](int k, int e) {
        if (st[(size_t)k] == AIR_OK) st[(size_t)k] = e;
    };
    if (cudaMallocHost((void **)&h_tab, 2 * nk * sizeof(AirConvJob)) != cudaSuccess ||
        cudaMalloc((void **)&d_tab, 2 * nk * sizeof(AirConvJob)) != cudaSuccess) {
        first = AIR_ERR_OOM;
    }
    for (auto &e : ev)
        if (first == AIR_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) first = AIR_ERR_CUDA;
    if (first != AIR_OK)
        for (int k = 0; k < count; ++k) fail(k, first);
    for (int k = 0; first == AIR_OK && k < count; ++k) {
        air_hierarchy *h = const_cast<air_hierarchy *>(H[k]);
        Hm[(size_t)k] = h;
        air_solve_info *inf = info ? &info[k] : &local[(size_t)k];
        if (!h || !b[k] || !x[k] || !(rtol > 0.0) || A[k].n_rows != h->lev[0].n) {
            fail(k, AIR_ERR_INVALID_ARG);
            continue;
        }
        if (streams && streams[k]) {
            str[(size_t)k] = (cudaStream_t)streams[k];
        } else if (cudaStreamCreateWithFlags(&own[(size_t)k], cudaStreamNonBlocking) == cudaSuccess) {
            str[(size_t)k] = own[(size_t)k];
        } else {
            fail(k, AIR_ERR_CUDA);
            continue;
        }
        cudaStream_t s = str[(size_t)k];
        AirCallStream call(s);
        const int64_t n = A[k].n_rows;
        if (A[k].on_device) {
            bd[(size_t)k] = b[k];
            xd[(size_t)k] = x[k];
        } else {
            // host vectors: the staging buffers of air_gmres_solve
            if (!h->lev[0].owns_A || h->lev[0].v == nullptr) {
                fail(k, AIR_ERR_INVALID_ARG);
                continue;
            }
            if (!h->bd && air_dmalloc((void **)&h->bd, (size_t)n * sizeof(double)) != cudaSuccess) fail(k, AIR_ERR_OOM);
            if (!h->xd && air_dmalloc((void **)&h->xd, (size_t)n * sizeof(double)) != cudaSuccess) fail(k, AIR_ERR_OOM);
            if (st[(size_t)k] != AIR_OK) continue;
            if (cudaMemcpyAsync(h->bd, b[k], (size_t)n * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess) {
                fail(k, AIR_ERR_CUDA);
                continue;
            }
            bd[(size_t)k] = h->bd;
            xd[(size_t)k] = h->xd;
        }
        const int e = air_gmres_open(g[(size_t)k], h->lev[0], h, bd[(size_t)k], xd[(size_t)k], rtol, s, inf);
        if (e != AIR_OK) fail(k, e);
    }
    auto live = [&](int k) { return st[(size_t)k] == AIR_OK && g[(size_t)k].phase != AirGmres::DONE; };
    auto sync_all = [&]() {
        for (int k = 0; k < count; ++k)
            if (str[(size_t)k] && cudaStreamSynchronize(str[(size_t)k]) != cudaSuccess) fail(k, AIR_ERR_CUDA);
    };
    if (first == AIR_OK) {
        sync_all();
        for (int k = 0; k < count; ++k)
            if (st[(size_t)k] == AIR_OK) air_gmres_after_open(g[(size_t)k]);
    }
    BatchVcycle bv;
    while (first == AIR_OK) {
        std::vector<int> members;
        bool stepping = false;
        for (int k = 0; k < count; ++k) {
            if (!live(k)) continue;
            members.push_back(k);
            stepping = stepping || g[(size_t)k].phase == AirGmres::STEP;
        }
        if (members.empty()) break;
        if (stepping) {
            if (members != bv.members || !bv.exec) {
                const int e = build_batch_vcycle(Hm, members, count, d_tab, d_tab + nk, &bv);
                if (e != AIR_OK) {
                    for (int k : members) fail(k, e);
                    break;
                }
            }
            for (int k = 0; k < count; ++k) {
                AirConvJob &in = h_tab[k], &out = h_tab[nk + (size_t)k];
                in = AirConvJob{nullptr, nullptr, 0, 0};
                out = AirConvJob{nullptr, nullptr, 0, 0};
                if (!live(k) || g[(size_t)k].phase != AirGmres::STEP) continue;
                const air_hierarchy *h = Hm[(size_t)k];
                const bool f64 = h->opt.precision == AIR_PREC_F64;
                in = AirConvJob{air_gmres_vj(g[(size_t)k]), h->lev[0].b, h->lev[0].n, f64 ? 0 : 1};
                out = AirConvJob{h->lev[0].x, air_gmres_zj(g[(size_t)k]), h->lev[0].n, f64 ? 0 : 2};
            }
            // the previous round's work on every stream is complete (synchronised)
            if (cudaMemcpyAsync(d_tab, h_tab, 2 * nk * sizeof(AirConvJob), cudaMemcpyHostToDevice, ms) != cudaSuccess ||
                cudaGraphLaunch(bv.exec, ms) != cudaSuccess || cudaEventRecord(ev[nk], ms) != cudaSuccess) {
                for (int k : members) fail(k, AIR_ERR_CUDA);
                break;
            }
            air_launch_counter_add(bv.kernels);
        }
        for (int k : members) {
            AirGmres &gk = g[(size_t)k];
            AirCallStream call(str[(size_t)k]);
            int e = AIR_OK;
            if (gk.phase == AirGmres::STEP) {
                if (cudaStreamWaitEvent(str[(size_t)k], ev[nk], 0) != cudaSuccess) e = AIR_ERR_CUDA;
                if (e == AIR_OK) e = air_gmres_step(gk);
            } else {
                e = air_gmres_cycle(gk);
            }
            if (e != AIR_OK) fail(k, e);
        }
        if (stepping && cudaStreamSynchronize(ms) != cudaSuccess) {
            for (int k : members) fail(k, AIR_ERR_CUDA);
            break;
        }
        sync_all();
        for (int k : members) {
            if (st[(size_t)k] != AIR_OK) continue;
            AirGmres &gk = g[(size_t)k];
            AirCallStream call(str[(size_t)k]);
            const int e = gk.phase == AirGmres::STEP ? air_gmres_after_step(gk) : air_gmres_after_cycle(gk);
            if (e != AIR_OK) fail(k, e);
        }
    }
    for (int k = 0; k < count; ++k) {
        int r = st[(size_t)k];
        if (r == AIR_OK && g[(size_t)k].H) {
            AirCallStream call(str[(size_t)k]);
            r = air_gmres_close(g[(size_t)k]);
            if (r >= 0 && !A[k].on_device) {
                const int64_t n = A[k].n_rows;
                if (cudaMemcpyAsync(x[k], xd[(size_t)k], (size_t)n * sizeof(double), cudaMemcpyDeviceToHost,
                                    str[(size_t)k]) != cudaSuccess ||
                    cudaStreamSynchronize(str[(size_t)k]) != cudaSuccess)
                    r = AIR_ERR_CUDA;
            }
        } else if (str[(size_t)k]) {
            cudaStreamSynchronize(str[(size_t)k]);
        }
        if (status) status[k] = r;
        if (first == AIR_OK && r < 0) first = r;
        if (own[(size_t)k]) cudaStreamDestroy(own[(size_t)k]);
    }
    for (auto e : ev)
        if (e) cudaEventDestroy(e);
    if (d_tab) cudaFree(d_tab);
    if (h_tab) cudaFreeHost(h_tab);
    cudaStreamDestroy(ms);
    return first;
}
