// Serving: continuous batching of independent multibody solves on one GPU.
//
// Requests are queued with their geometry and boundary data.  A scheduler
// admits them whenever a slot is free and the request's estimated device
// footprint fits in the remaining HBM budget, in arrival order or (policy 1)
// shortest estimated work first; every admitted request runs its whole
// pipeline (S build, right-hand side, mixed-precision or FP64 solve) on its
// own context and CUDA stream, so the work of concurrent requests overlaps on
// the device.  Finished requests release their memory and slot, which admits
// the next ones.  A request's launch shapes depend only on its own sizes, so
// its result is the same alone and in a mix.  Each request records CUDA
// events on its stream around its work and times its G_hat launches, so the
// device-side overlap of requests can be measured.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

struct Req {
    int64_t id;
    int dim;
    double kappa;
    std::vector<mbs_shape> shapes;
    std::vector<std::vector<double>> pts;  // x, y, z per shape (3 vectors each)
    std::vector<mbs_body> bodies;
    int nrhs;
    std::vector<double> v;
    double tol;
    int fp64 = 0;
    int max_iter = 0;
    size_t footprint;
    double work = 0.0;  // estimated device work (policy 1)
    mbs_request_result res;
    std::vector<double> qhat;
};

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// Upper estimate of the device bytes one request holds while it runs.
size_t estimate_footprint(const Req& r, int restart) {
    size_t N = 0, M = 0, shape_bytes = 0, work = 0;
    std::vector<char> used(r.shapes.size(), 0);
    for (const auto& b : r.bodies) used[b.shape] = 1;
    for (size_t s = 0; s < r.shapes.size(); ++s) {
        if (!used[s]) continue;
        const mbs_shape& sh = r.shapes[s];
        const size_t kc = sh.k > 0 ? sh.k : std::min(sh.m, sh.p);
        const size_t mp = std::min(sh.p, sh.m);
        // kept: A | U, Z*, C, S (FP64 and FP32), the SVD factors of A (two n x n)
        shape_bytes += 16 * ((size_t)sh.m * (sh.n + kc) + kc * sh.m + (size_t)sh.m * sh.n + kc * kc +
                             2 * (size_t)sh.n * sh.n) + 8 * kc * kc;
        // build work space: B | D, W1, W2, W3, R_B^H, R_A^H and vectors
        work += 16 * ((size_t)sh.p * (sh.m + sh.n) + kc * std::max(sh.m, sh.n) + mp * sh.n + (size_t)sh.m * sh.n +
                      (size_t)sh.m * mp + (size_t)sh.n * sh.n) + 64 * (sh.p + sh.m + sh.n);
    }
    for (const auto& b : r.bodies) {
        const mbs_shape& sh = r.shapes[b.shape];
        N += sh.k > 0 ? sh.k : std::min(sh.m, sh.p);
        M += sh.m;
    }
    const size_t T = r.bodies.size();
    const size_t nr = r.nrhs;
    size_t bytes = shape_bytes + std::min(work, (size_t)8 << 30);
    bytes += T * T * 20 + N * 40;
    bytes += (size_t)(restart + 1) * N * nr * 8;  // FP32 Krylov basis
    bytes += N * nr * (16 * 8 + 8 * 6);           // FP64/FP32 vectors, partial sums (<= 64 splits chunked)
    bytes += (size_t)64 * N * nr * 16;            // split partials upper bound
    bytes += M * nr * 16;
    return bytes + ((size_t)64 << 20);
}

// Estimated device work of one request for shortest-work-first admission:
// G_hat pairs per application (the number of applications is not known in
// advance, so per-application cost stands for it) plus the S build's cubic
// terms.
double estimate_work(const Req& r) {
    double N = 0.0, sq = 0.0, build = 0.0;
    std::vector<char> used(r.shapes.size(), 0);
    for (const auto& b : r.bodies) {
        const mbs_shape& sh = r.shapes[b.shape];
        const double k = sh.k > 0 ? sh.k : std::min(sh.m, sh.p);
        N += k;
        sq += k * k;
        if (!used[b.shape]) {
            used[b.shape] = 1;
            build += (double)sh.p * (sh.m + sh.n) * std::min(sh.p, sh.m);
        }
    }
    return (N * N - sq) * r.nrhs + 64.0 * build;
}

}  // namespace

struct mbs_server {
    int max_active = 1;
    size_t budget = 0;
    size_t in_use = 0;
    int active = 0;
    int64_t next_id = 1;
    int policy = 0;  // 0 arrival order, 1 shortest estimated work first
    bool stop = false;
    cudaEvent_t base = nullptr;  // device clock origin of the request timings
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Req>> queue;
    std::map<int64_t, std::shared_ptr<Req>> all;
    std::vector<std::thread> workers;
    int device = 0;
};

namespace {

void run_request(mbs_server* srv, std::shared_ptr<Req> r) {
    cudaSetDevice(srv->device);
    mbs_options o;
    mbs_default_options(&o);
    o.precision = r->fp64 ? MBS_PREC_FP64 : MBS_PREC_MIXED;
    o.tol = r->tol;
    if (r->max_iter > 0) o.max_iter = r->max_iter;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    mbs_status st = MBS_OK;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        st = MBS_ERR_CUDA;
    }
    o.stream = s;
    mbs_ctx* c = nullptr;
    if (st == MBS_OK) st = mbs_create(r->dim, r->kappa, &o, &c);
    if (st == MBS_OK) st = mbs_profile(c, 1);
    int64_t N = 0;
    mbs_solve_info info;
    std::memset(&info, 0, sizeof(info));
    std::vector<double> b;
    double kt[7] = {0, 0, 0, 0, 0, 0, 0};
    if (st == MBS_OK && cudaEventRecord(e0, s) != cudaSuccess) st = MBS_ERR_CUDA;
    if (st == MBS_OK)
        st = mbs_build_scattering_matrices(c, (int)r->shapes.size(), r->shapes.data(),
                                           (int)r->bodies.size(), r->bodies.data());
    if (st == MBS_OK) st = mbs_get_layout(c, &N, nullptr, nullptr);
    if (st == MBS_OK) {
        b.assign((size_t)2 * N * r->nrhs, 0.0);
        st = mbs_rhs(c, r->nrhs, r->v.data(), b.data());
    }
    bool capped = false;
    if (st == MBS_OK) {
        r->qhat.assign((size_t)2 * N * r->nrhs, 0.0);
        st = mbs_solve(c, r->nrhs, b.data(), r->qhat.data(), &info);
        // an iteration cap set by the request ends the solve without an error
        if (st == MBS_ERR_NOCONV && r->max_iter > 0) {
            st = MBS_OK;
            capped = true;
        }
    }
    double dev0 = 0.0, dev1 = 0.0;
    if (st == MBS_OK && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess) {
        float a = 0.f, z = 0.f;
        if (cudaEventElapsedTime(&a, srv->base, e0) == cudaSuccess &&
            cudaEventElapsedTime(&z, srv->base, e1) == cudaSuccess) {
            dev0 = 1e-3 * a;
            dev1 = 1e-3 * z;
        }
        mbs_kernel_times(c, kt);
    }
    cudaGetLastError();
    mbs_destroy(c);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    std::lock_guard<std::mutex> g(srv->mu);
    r->res.status = st;
    r->res.N = N;
    r->res.rel_residual = info.rel_residual;
    r->res.inner_iterations = info.inner_iterations;
    r->res.converged = (st == MBS_OK && !capped && info.converged) ? 1 : 0;
    r->res.dev_start = dev0;
    r->res.dev_end = dev1;
    r->res.g_busy_ms = kt[0] + kt[2];
    r->res.t_end = now_s();
    r->res.done = (st == MBS_OK) ? 1 : -1;
    srv->in_use -= r->footprint;
    srv->active--;
    srv->cv.notify_all();
}

void worker_loop(mbs_server* srv) {
    cudaSetDevice(srv->device);
    while (true) {
        std::shared_ptr<Req> r;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            // the candidate: the head of the queue (arrival order) or the queued
            // request of least estimated work (ties: the earlier one)
            auto pick = [&]() -> std::deque<std::shared_ptr<Req>>::iterator {
                auto best = srv->queue.begin();
                if (srv->policy == 1)
                    for (auto it = srv->queue.begin(); it != srv->queue.end(); ++it)
                        if ((*it)->work < (*best)->work) best = it;
                return best;
            };
            srv->cv.wait(lk, [&] {
                if (srv->stop) return true;
                if (srv->queue.empty()) return false;
                const auto& cand = *pick();
                // admission: a free slot and room for the candidate; an oversized
                // request runs alone.
                return srv->active == 0 ||
                       (srv->active < srv->max_active && srv->in_use + cand->footprint <= srv->budget);
            });
            if (srv->stop && srv->queue.empty()) return;
            if (srv->queue.empty()) continue;
            auto it = pick();
            r = *it;
            srv->queue.erase(it);
            srv->active++;
            srv->in_use += r->footprint;
            r->res.t_start = now_s();
        }
        run_request(srv, r);
    }
}

}  // namespace

extern "C" {

mbs_status mbs_serve_create(int max_active, size_t hbm_budget, mbs_server** out) {
    if (!out || max_active < 1) return MBS_ERR_ARG;
    *out = nullptr;
    mbs_server* s = new mbs_server();
    s->max_active = max_active;
    cudaGetDevice(&s->device);
    if (hbm_budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return MBS_ERR_CUDA;
        }
        hbm_budget = (size_t)(0.9 * (double)fr);
    }
    s->budget = hbm_budget;
    if (cudaEventCreate(&s->base) != cudaSuccess || cudaEventRecord(s->base, 0) != cudaSuccess ||
        cudaEventSynchronize(s->base) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return MBS_ERR_CUDA;
    }
    for (int i = 0; i < max_active; ++i) s->workers.emplace_back(worker_loop, s);
    *out = s;
    return MBS_OK;
}

mbs_status mbs_serve_submit(mbs_server* srv, const mbs_request* q, int64_t* id) {
    if (!srv || !q || !id || (q->dim != 2 && q->dim != 3) || q->nshapes < 1 || q->nbodies < 1 ||
        q->nrhs < 1 || !q->shapes || !q->bodies || !q->v || !(q->kappa > 0) || !(q->tol > 0))
        return MBS_ERR_ARG;
    auto r = std::make_shared<Req>();
    r->dim = q->dim;
    r->kappa = q->kappa;
    r->nrhs = q->nrhs;
    r->tol = q->tol;
    r->fp64 = q->fp64 ? 1 : 0;
    r->max_iter = q->max_iter > 0 ? q->max_iter : 0;
    r->shapes.assign(q->shapes, q->shapes + q->nshapes);
    r->pts.resize((size_t)3 * q->nshapes);
    size_t M = 0;
    for (int s = 0; s < q->nshapes; ++s) {
        mbs_shape& sh = r->shapes[s];
        if (sh.m < 2 || sh.n < 1 || sh.p < 1 || !sh.x || !sh.y || !sh.z) return MBS_ERR_ARG;
        r->pts[3 * s].assign(sh.x, sh.x + (size_t)q->dim * sh.m);
        r->pts[3 * s + 1].assign(sh.y, sh.y + (size_t)q->dim * sh.n);
        r->pts[3 * s + 2].assign(sh.z, sh.z + (size_t)q->dim * sh.p);
        sh.x = r->pts[3 * s].data();
        sh.y = r->pts[3 * s + 1].data();
        sh.z = r->pts[3 * s + 2].data();
    }
    r->bodies.assign(q->bodies, q->bodies + q->nbodies);
    for (const auto& b : r->bodies) {
        if (b.shape < 0 || b.shape >= q->nshapes) return MBS_ERR_ARG;
        M += r->shapes[b.shape].m;
    }
    r->v.assign(q->v, q->v + 2 * M * q->nrhs);
    mbs_options o;
    mbs_default_options(&o);
    r->footprint = estimate_footprint(*r, o.restart);
    r->work = estimate_work(*r);
    std::memset(&r->res, 0, sizeof(r->res));
    {
        std::lock_guard<std::mutex> g(srv->mu);
        r->id = srv->next_id++;
        r->res.t_submit = now_s();
        srv->all[r->id] = r;
        srv->queue.push_back(r);
        *id = r->id;
    }
    srv->cv.notify_all();
    return MBS_OK;
}

mbs_status mbs_serve_poll(mbs_server* srv, int64_t id, mbs_request_result* res, double* qhat) {
    if (!srv || !res) return MBS_ERR_ARG;
    std::lock_guard<std::mutex> g(srv->mu);
    auto it = srv->all.find(id);
    if (it == srv->all.end()) return MBS_ERR_ARG;
    *res = it->second->res;
    if (qhat && it->second->res.done == 1)
        std::memcpy(qhat, it->second->qhat.data(), it->second->qhat.size() * sizeof(double));
    return MBS_OK;
}

mbs_status mbs_serve_set_policy(mbs_server* srv, int policy) {
    if (!srv || policy < 0 || policy > 1) return MBS_ERR_ARG;
    std::lock_guard<std::mutex> g(srv->mu);
    srv->policy = policy;
    return MBS_OK;
}

mbs_status mbs_serve_drain(mbs_server* srv) {
    if (!srv) return MBS_ERR_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    srv->cv.wait(lk, [&] { return srv->queue.empty() && srv->active == 0; });
    return MBS_OK;
}

void mbs_serve_destroy(mbs_server* srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->stop = true;
    }
    srv->cv.notify_all();
    for (auto& t : srv->workers) t.join();
    if (srv->base) cudaEventDestroy(srv->base);
    delete srv;
}

}  // extern "C"
