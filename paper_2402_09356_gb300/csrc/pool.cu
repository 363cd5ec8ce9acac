// Worker pool over the likelihood path (include/tlr.h, "many datasets"):
// resident datasets, requests admitted under an HBM budget (sched.cuh) and
// evaluated by concurrent workers, each a host thread with its own context
// and stream.  Every evaluation is an ordinary tlr_loglik call on the
// dataset's own factor storage, started from the dataset's own rank map.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "common.cuh"
#include "compress.cuh"
#include "sched.cuh"
#include "tlr_internal.cuh"

namespace tlr {
namespace {

thread_local std::string t_pool_err;

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// Device bytes of a dataset's factor storage: compact slots from its rank
// map when it has one (plan_slots), else uniform maxrank slots.
int64_t factor_bytes(int64_t n, int nb, int maxrank, const std::vector<int32_t> &hint) {
    tlr_mat M;
    M.n = n;
    M.nb = nb;
    M.nt = (int)ceil_div(n, nb);
    M.maxrank = maxrank;
    const int64_t cols = plan_slots(&M, hint), nt = M.nt;
    return (nt * nb * nb + 2 * cols * nb) * 8 + nt * nt * 4;
}

// Estimated device workspace of one evaluation (allocated inside it): the two
// panel buffers and the paired-FP32 panel, the compression buffers of one
// column (5 m s + 7 s^2 doubles per tile at the largest sample size s), the
// Gram matrices G_k = V_k' V_k of the finished columns (S_k^2 doubles, S_k the
// summed ranks of column k, +25%), and 64 MiB of small buffers.  Ranks come
// from the dataset's last factor; before the first evaluation every rank is
// taken as min(maxrank, 64).
int64_t work_bytes(int64_t n, int nb, int maxrank, const std::vector<int32_t> &hint) {
    const int nt = (int)ceil_div(n, nb);
    const bool have = hint.size() == (size_t)nt * nt;
    int rmax = 0;
    double gram = 0.0;
    for (int k = 0; k < nt; ++k) {
        double S = 0.0;
        for (int i = k + 1; i < nt; ++i) {
            int r = have ? hint[(size_t)i * nt + k] : std::min(maxrank, 64);
            S += r;
            rmax = std::max(rmax, r);
        }
        gram += S * S * 8.0;
    }
    if (!have) rmax = maxrank;
    const int64_t s = std::min<int64_t>(rmax + 32, kMaxSample);
    const int64_t panel = 3 * (int64_t)nt * nb * nb * 8;
    const int64_t comp = (int64_t)nt * (5 * nb * s + 7 * s * s) * 8;
    return panel + comp + (int64_t)(1.25 * gram) + ((int64_t)64 << 20);
}

struct PoolData {
    int id = -1;
    int64_t n = 0;
    int nb = 0, maxrank = 0;
    double *xy = nullptr, *z = nullptr;
    int64_t *perm = nullptr;
    std::vector<int32_t> hint;  // rank map of the last factor (empty before the first)
    double pivot2 = 0.0;        // min L_ii^2 / sigma2 of the last likelihood (auto precision)
    tlr_mat *L = nullptr;       // resident factor storage (null while evicted)
    int queued = 0;             // submitted, not finished
    bool removing = false;
};

struct PoolReq {
    int64_t ticket = 0;
    int id = -1;
    tlr_theta theta{};
    double eps = 0.0;
    int precision = TLR_PREC_FP64;
    Clock::time_point t_submit, t_start, t_done;
    bool done = false;
    int status = TLR_OK;
    std::string err;
    tlr_result res{};
};

struct Worker {
    tlr_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
};

// Tuning of a pool (tlr_pool_configure): requests a worker evaluates
// together, and the rank buckets of every worker's context.
struct PoolConfig {
    int group = 1;
    tlr_buckets buckets = default_buckets();
};

int pool_fail(int code, const std::string &msg) {
    t_pool_err = msg;
    return code;
}

}  // namespace
}  // namespace tlr

using namespace tlr;

struct tlr_pool {
    int device = 0;
    tlr_pool_opts opts{};
    cudaMemPool_t mp = nullptr;  // factor storage and resident data
    tlr_ctx *ctl = nullptr;      // ordering of added datasets
    cudaStream_t ctl_stream = nullptr;
    std::mutex ctl_mu;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    Admission adm;
    std::unordered_map<int, std::unique_ptr<PoolData>> data;
    std::unordered_map<int64_t, std::unique_ptr<PoolReq>> reqs;
    int64_t next_ticket = 1;
    int64_t completed = 0, running = 0, max_running = 0, allocations = 0, resident_bytes = 0;
    int64_t groups = 0, grouped = 0;  // group evaluations run, requests they held
    PoolConfig cfg;
    std::vector<Worker> workers;
    std::vector<std::thread> threads;
};

namespace {

// TLR matrix storage from the pool's memory pool, stream ordered on s, zeroed
// like tlr_mat_create's: compact slots from `hint` when given, else uniform.
tlr_mat *mat_alloc(tlr_pool *p, int64_t n, int nb, int maxrank, const std::vector<int32_t> &hint, cudaStream_t s) {
    auto *M = new tlr_mat();
    M->device = p->device;
    M->n = n;
    M->nb = nb;
    M->nt = (int)ceil_div(n, nb);
    M->maxrank = maxrank;
    const int64_t cols = plan_slots(M, hint);
    const size_t db = (size_t)M->nt * nb * nb * sizeof(double);
    const size_t ub = (size_t)cols * nb * sizeof(double);
    const size_t rb = (size_t)M->nt * M->nt * sizeof(int32_t);
    M->bytes = db + 2 * ub + rb;
    cudaError_t e = cudaMallocFromPoolAsync((void **)&M->D, db, p->mp, s);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void **)&M->U, ub, p->mp, s);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void **)&M->V, ub, p->mp, s);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void **)&M->ranks, rb, p->mp, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(M->D, 0, db, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(M->U, 0, ub, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(M->V, 0, ub, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(M->ranks, 0, rb, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (void *q : {(void *)M->D, (void *)M->U, (void *)M->V, (void *)M->ranks})
            if (q) cudaFreeAsync(q, s);
        delete M;
        return nullptr;
    }
    return M;
}

void mat_free(tlr_mat *M, cudaStream_t s) {
    if (!M) return;
    for (void *q : {(void *)M->D, (void *)M->U, (void *)M->V, (void *)M->ranks})
        if (q) cudaFreeAsync(q, s);
    delete M;
}

// One admitted request of a worker's group.
struct Run {
    Admission::Req ar{};
    bool alloc = false;
    PoolReq *r = nullptr;
    PoolData *d = nullptr;
    std::vector<tlr_mat *> to_free;
    int status = TLR_OK;
    std::string err;
    std::vector<int32_t> hint;
    bool ran = false;
    int64_t extra = 0;  // storage charged for a retry on uniform slots
    double pivot2 = 0.0;
    tlr_opts o{};
};

void worker_main(tlr_pool *p, int w) {
    Worker &W = p->workers[(size_t)w];
    cudaSetDevice(p->device);
    std::unique_lock<std::mutex> lk(p->mu);
    for (;;) {
        std::vector<Run> runs(1);
        std::vector<int> evicted;
        while (!p->adm.admit(&runs[0].ar, &runs[0].alloc, &evicted)) {
            if (p->stop && p->adm.queued() == 0) return;
            p->cv_work.wait(lk);
        }
        // companions: queued requests of the same precision that can start
        // now, evaluated together with the first (tlr_loglik_batch)
        const PoolConfig cfg = p->cfg;
        const int prec = p->reqs[runs[0].ar.ticket]->precision;
        auto same_path = [&](const Admission::Req &q) { return p->reqs[q.ticket]->precision == prec; };
        for (;;) {
            if ((int)runs.size() >= cfg.group) break;
            Run next;
            if (!p->adm.admit(&next.ar, &next.alloc, &evicted, same_path)) break;
            runs.push_back(std::move(next));
        }
        for (Run &u : runs) {
            u.r = p->reqs[u.ar.ticket].get();
            u.d = p->data[u.ar.data].get();
            u.r->t_start = Clock::now();
            p->max_running = std::max(p->max_running, ++p->running);
            if (u.alloc) ++p->allocations;
        }
        std::vector<tlr_mat *> to_free;
        for (int e : evicted) {
            PoolData *v = p->data[e].get();
            to_free.push_back(v->L);
            v->L = nullptr;
        }
        lk.unlock();

        // The evicted factors' last requests have finished (their workers
        // synced), so their storage is free to go on this worker's stream.
        for (tlr_mat *M : to_free) mat_free(M, W.stream);
        W.ctx->buckets = cfg.buckets;
        for (Run &u : runs) {
            PoolData *d = u.d;
            if (u.alloc && !d->L) d->L = mat_alloc(p, d->n, d->nb, d->maxrank, d->hint, W.stream);
            u.o.nb = d->nb;
            u.o.maxrank = d->maxrank;
            u.o.eps = u.r->eps;
            u.o.precision = u.r->precision;
            u.pivot2 = d->pivot2;
            if (!d->L) {
                u.status = TLR_ERR_OOM;
                u.err = "cannot allocate the factor storage of dataset " + std::to_string(d->id);
            }
        }
        auto evaluate = [&](Run &u, tlr_mat *M) {
            PoolData *d = u.d;
            M->h_ranks = d->hint;
            M->last_pivot2 = d->pivot2;
            u.status = tlr_loglik(W.ctx, d->xy, d->z, d->n, u.r->theta, &u.o, M, &u.r->res, W.stream);
            u.err = u.status != TLR_OK ? std::string(tlr_last_error(W.ctx)) : std::string();
            u.hint = M->h_ranks;
            u.pivot2 = M->last_pivot2;
            u.ran = true;
        };
        {
            std::vector<Run *> go;
            for (Run &u : runs)
                if (u.d->L) go.push_back(&u);
            if (go.size() == 1) {
                evaluate(*go[0], go[0]->d->L);
            } else if (go.size() > 1) {
                std::vector<BatchEntry> es;
                for (Run *u : go) {
                    PoolData *d = u->d;
                    d->L->h_ranks = d->hint;
                    d->L->last_pivot2 = d->pivot2;
                    BatchEntry e;
                    e.xy = d->xy;
                    e.z = d->z;
                    e.n = d->n;
                    e.theta = u->r->theta;
                    e.opts = &u->o;
                    e.L = d->L;
                    e.out = &u->r->res;
                    es.push_back(e);
                }
                int call = TLR_OK;
                std::string call_err;
                try {
                    loglik_batch(W.ctx, es, W.stream);
                } catch (const Error &e) {
                    call = e.code;
                    call_err = e.msg;
                } catch (const std::exception &e) {
                    call = TLR_ERR_CUDA;
                    call_err = e.what();
                }
                for (size_t g = 0; g < go.size(); ++g) {
                    Run &u = *go[g];
                    u.status = call != TLR_OK ? call : es[g].status;
                    u.err = call != TLR_OK ? call_err : es[g].msg;
                    u.hint = u.d->L->h_ranks;
                    u.pivot2 = u.d->L->last_pivot2;
                    u.ran = true;
                }
            }
        }
        for (Run &u : runs) {
            PoolData *d = u.d;
            if (!(d->L && u.status == TLR_ERR_RANK && d->L->cap_overflow)) continue;
            // the compact slots (sized by the last rank map) ran out of
            // room: the same evaluation, from the same rank map, on
            // uniform maxrank slots (held only for this request).  The
            // difference in storage is charged to the budget first,
            // waiting for running requests or evicting idle factors.
            const int64_t need = factor_bytes(d->n, d->nb, d->maxrank, {}) - (int64_t)d->L->bytes;
            std::vector<int> ev2;
            bool never = false, got = false;
            std::vector<tlr_mat *> free2;
            lk.lock();
            while (!(got = p->adm.grow(u.ar.data, need, &ev2, &never)) && !never) p->cv_done.wait(lk);
            for (int e : ev2) {
                PoolData *v = p->data[e].get();
                free2.push_back(v->L);
                v->L = nullptr;
            }
            lk.unlock();
            for (tlr_mat *M : free2) mat_free(M, W.stream);
            if (got) {
                u.extra = std::max<int64_t>(need, 0);
                mat_free(d->L, W.stream);
                d->L = mat_alloc(p, d->n, d->nb, d->maxrank, {}, W.stream);
                if (d->L) {
                    evaluate(u, d->L);
                } else {
                    u.status = TLR_ERR_OOM;
                    u.err = "cannot allocate uniform factor storage after a slot overflow";
                }
            } else {
                u.status = TLR_ERR_OOM;
                u.err = "uniform factor storage after a slot overflow exceeds the HBM budget";
            }
        }
        std::vector<int64_t> wb(runs.size()), fb(runs.size());
        for (size_t q = 0; q < runs.size(); ++q) {
            Run &u = runs[q];
            PoolData *d = u.d;
            // uniform storage (first request, or after an overflow) is given back;
            // the next request allocates compact slots from the new rank map
            tlr_mat *drop = (d->L && d->L->base_off.empty()) ? d->L : nullptr;
            if (drop) {
                mat_free(drop, W.stream);
                d->L = nullptr;
            }
            const std::vector<int32_t> &nh = u.ran ? u.hint : d->hint;
            wb[q] = work_bytes(d->n, d->nb, d->maxrank, nh);
            fb[q] = factor_bytes(d->n, d->nb, d->maxrank, nh);
        }

        lk.lock();
        for (size_t q = 0; q < runs.size(); ++q) {
            Run &u = runs[q];
            PoolData *d = u.d;
            if (u.ran) {
                d->hint.swap(u.hint);
                d->pivot2 = u.pivot2;
            }
            p->adm.shrink(u.extra);
            p->adm.finish(u.ar.data, d->L != nullptr);
            p->adm.set_work(u.ar.data, wb[q]);
            if (!d->L) p->adm.set_factor(u.ar.data, fb[q]);
            u.r->status = u.status;
            u.r->err = u.err;
            u.r->t_done = Clock::now();
            u.r->done = true;
            --d->queued;
            --p->running;
            ++p->completed;
        }
        if (runs.size() > 1) {
            ++p->groups;
            p->grouped += (int64_t)runs.size();
        }
        p->cv_done.notify_all();
        p->cv_work.notify_all();
    }
}

PoolData *find_data(tlr_pool *p, int id) {
    auto it = p->data.find(id);
    return it == p->data.end() || it->second->removing ? nullptr : it->second.get();
}

// Blocks (lock held) until dataset d has no queued or running request.
void wait_idle(tlr_pool *p, std::unique_lock<std::mutex> &lk, PoolData *d) {
    p->cv_done.wait(lk, [&] { return d->queued == 0; });
}

int submit_locked(tlr_pool *p, PoolData *d, tlr_theta th, double eps, int prec, int64_t *ticket) {
    auto r = std::make_unique<PoolReq>();
    r->ticket = p->next_ticket++;
    r->id = d->id;
    r->theta = th;
    r->eps = eps;
    r->precision = prec;
    r->t_submit = Clock::now();
    *ticket = r->ticket;
    p->adm.enqueue(r->ticket, d->id);
    ++d->queued;
    p->reqs.emplace(r->ticket, std::move(r));
    p->cv_work.notify_one();
    return TLR_OK;
}

int wait_locked(tlr_pool *p, std::unique_lock<std::mutex> &lk, int64_t ticket, tlr_result *out, double *times) {
    auto it = p->reqs.find(ticket);
    if (it == p->reqs.end()) return pool_fail(TLR_ERR_ARG, "unknown ticket " + std::to_string(ticket));
    PoolReq *r = it->second.get();
    p->cv_done.wait(lk, [&] { return r->done; });
    if (out) *out = r->res;
    if (times) {
        times[0] = ms_between(r->t_submit, r->t_start);
        times[1] = ms_between(r->t_start, r->t_done);
        times[2] = ms_between(r->t_submit, r->t_done);
    }
    int st = r->status;
    if (st != TLR_OK) t_pool_err = r->err;
    p->reqs.erase(it);
    return st;
}

bool args_ok(double eps, int prec) {
    return eps >= 0 && std::isfinite(eps) &&
           (prec == TLR_PREC_FP64 || prec == TLR_PREC_MIXED || prec == TLR_PREC_AUTO || prec == TLR_PREC_TENSOR);
}

}  // namespace

extern "C" {

const char *tlr_pool_last_error(void) { return t_pool_err.c_str(); }

int tlr_pool_create(int device, const tlr_pool_opts *opts, tlr_pool **out) {
    if (!out || !opts) return pool_fail(TLR_ERR_ARG, "opts/out");
    *out = nullptr;
    if (opts->workers < 1 || opts->workers > 64) return pool_fail(TLR_ERR_ARG, "workers must be 1..64");
    if (opts->nb < 16 || opts->nb > kMaxTile) return pool_fail(TLR_ERR_ARG, "nb must be 16..1024");
    if (opts->flags != 0) return pool_fail(TLR_ERR_ARG, "flags");
    auto *p = new tlr_pool();
    p->device = device;
    p->opts = *opts;
    auto cleanup = [&](int code, const std::string &msg) {
        tlr_pool_destroy(p);
        return pool_fail(code, msg);
    };
    int rc = tlr_ctx_create(device, &p->ctl);
    if (rc != TLR_OK) return cleanup(rc, "cannot create a context on device " + std::to_string(device));
    if (cudaStreamCreateWithFlags(&p->ctl_stream, cudaStreamNonBlocking) != cudaSuccess)
        return cleanup(TLR_ERR_CUDA, "cannot create a stream");
    p->workers.resize((size_t)opts->workers);
    for (Worker &W : p->workers) {
        rc = tlr_ctx_create(device, &W.ctx);
        if (rc != TLR_OK) return cleanup(rc, "cannot create a worker context");
        // several factorisations share the SMs: no look-ahead shared-memory
        // reservation (it would hold every SM to one look-ahead CTA in total)
        if (opts->workers > 1) W.ctx->ahead_ctas_per_sm = 0;
        if (cudaStreamCreateWithFlags(&W.stream, cudaStreamNonBlocking) != cudaSuccess)
            return cleanup(TLR_ERR_CUDA, "cannot create a worker stream");
    }
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&p->mp, &props) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(TLR_ERR_CUDA, "cannot create a memory pool");
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return cleanup(TLR_ERR_CUDA, "cudaMemGetInfo");
    int64_t budget = opts->hbm_budget > 0 ? opts->hbm_budget : (int64_t)(0.9 * (double)free_b);
    // freed factor storage stays in the pool for the next allocation
    uint64_t keep = (uint64_t)budget;
    cudaMemPoolSetAttribute(p->mp, cudaMemPoolAttrReleaseThreshold, &keep);
    p->adm = Admission(budget);
    for (int w = 0; w < opts->workers; ++w) p->threads.emplace_back(worker_main, p, w);
    *out = p;
    return TLR_OK;
}

void tlr_pool_destroy(tlr_pool *p) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(p->mu);
        p->stop = true;
    }
    p->cv_work.notify_all();
    for (std::thread &t : p->threads) t.join();
    cudaSetDevice(p->device);
    for (auto &kv : p->data) {
        PoolData *d = kv.second.get();
        mat_free(d->L, p->ctl_stream);
        for (void *q : {(void *)d->xy, (void *)d->z, (void *)d->perm})
            if (q) cudaFreeAsync(q, p->ctl_stream);
    }
    if (p->ctl_stream) cudaStreamSynchronize(p->ctl_stream);
    for (Worker &W : p->workers) {
        if (W.stream) cudaStreamDestroy(W.stream);
        tlr_ctx_destroy(W.ctx);
    }
    if (p->ctl_stream) cudaStreamDestroy(p->ctl_stream);
    tlr_ctx_destroy(p->ctl);
    if (p->mp) cudaMemPoolDestroy(p->mp);
    delete p;
}

int tlr_pool_add(tlr_pool *p, const double *xy, const double *z, int64_t n, int order, uint64_t seed, int nb,
                 int *id) {
    if (!p || !xy || !z || !id) return pool_fail(TLR_ERR_ARG, "pool/xy/z/id");
    if (n <= 0 || n >= ((int64_t)1 << 31)) return pool_fail(TLR_ERR_ARG, "n");
    if (order < TLR_ORDER_IDENTITY || order > TLR_ORDER_MAXMIN) return pool_fail(TLR_ERR_ARG, "order");
    if (nb <= 0) nb = p->opts.nb;
    if (nb < 16 || nb > kMaxTile) return pool_fail(TLR_ERR_ARG, "nb must be 16..1024");
    const int maxrank = p->opts.maxrank > 0 ? std::min(p->opts.maxrank, nb) : nb / 2;
    const int64_t base = n * 32;  // locations (2n), observations, permutation
    const int64_t fb = factor_bytes(n, nb, maxrank, {}), wb = work_bytes(n, nb, maxrank, {});
    int slot;
    {
        std::lock_guard<std::mutex> lk(p->mu);
        if (!p->adm.can_add(base, fb, wb))
            return pool_fail(TLR_ERR_OOM, "dataset of n = " + std::to_string(n) +
                                              " does not fit the pool's HBM budget beside the others");
        slot = p->adm.add(base, fb, wb);  // reserves its bytes now
    }
    auto d = std::make_unique<PoolData>();
    d->id = slot;
    d->n = n;
    d->nb = nb;
    d->maxrank = maxrank;
    int rc = TLR_OK;
    std::string err;
    {
        std::lock_guard<std::mutex> cl(p->ctl_mu);
        cudaStream_t s = p->ctl_stream;
        double *xy_in = nullptr, *z_in = nullptr;
        cudaError_t e = cudaMallocFromPoolAsync((void **)&d->xy, (size_t)2 * n * 8, p->mp, s);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void **)&d->z, (size_t)n * 8, p->mp, s);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void **)&d->perm, (size_t)n * 8, p->mp, s);
        if (e == cudaSuccess) e = cudaMallocAsync((void **)&xy_in, (size_t)2 * n * 8, s);
        if (e == cudaSuccess) e = cudaMallocAsync((void **)&z_in, (size_t)n * 8, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(xy_in, xy, (size_t)2 * n * 8, cudaMemcpyDefault, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(z_in, z, (size_t)n * 8, cudaMemcpyDefault, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = e == cudaErrorMemoryAllocation ? TLR_ERR_OOM : TLR_ERR_CUDA;
            err = std::string("dataset upload: ") + cudaGetErrorString(e);
        } else {
            rc = tlr_order(p->ctl, xy_in, n, order, seed, 0, d->perm, nullptr, d->xy, s);
            if (rc == TLR_OK) rc = tlr_gather(p->ctl, d->perm, z_in, n, d->z, s);
            if (rc != TLR_OK) err = tlr_last_error(p->ctl);
        }
        if (xy_in) cudaFreeAsync(xy_in, s);
        if (z_in) cudaFreeAsync(z_in, s);
        if (cudaStreamSynchronize(s) != cudaSuccess && rc == TLR_OK) {
            rc = TLR_ERR_CUDA;
            err = "dataset upload: stream sync failed";
        }
        if (rc != TLR_OK) {
            for (void *q : {(void *)d->xy, (void *)d->z, (void *)d->perm})
                if (q) cudaFreeAsync(q, s);
            cudaStreamSynchronize(s);
        }
    }
    std::lock_guard<std::mutex> lk(p->mu);
    if (rc != TLR_OK) {
        p->adm.remove(slot);
        return pool_fail(rc, err);
    }
    p->resident_bytes += base;
    p->data.emplace(slot, std::move(d));
    *id = slot;
    return TLR_OK;
}

int tlr_pool_remove(tlr_pool *p, int id) {
    if (!p) return pool_fail(TLR_ERR_ARG, "pool");
    std::unique_ptr<PoolData> d;
    {
        std::unique_lock<std::mutex> lk(p->mu);
        PoolData *x = find_data(p, id);
        if (!x) return pool_fail(TLR_ERR_ARG, "unknown dataset " + std::to_string(id));
        x->removing = true;
        wait_idle(p, lk, x);
        p->adm.remove(id);
        p->resident_bytes -= x->n * 32;
        d = std::move(p->data[id]);
        p->data.erase(id);
    }
    std::lock_guard<std::mutex> cl(p->ctl_mu);
    mat_free(d->L, p->ctl_stream);
    for (void *q : {(void *)d->xy, (void *)d->z, (void *)d->perm})
        if (q) cudaFreeAsync(q, p->ctl_stream);
    cudaStreamSynchronize(p->ctl_stream);
    return TLR_OK;
}

int tlr_pool_dataset(tlr_pool *p, int id, int64_t *n, int *nb, const double **xy, const double **z,
                     const int64_t **perm, int32_t *last_max_rank) {
    if (!p) return pool_fail(TLR_ERR_ARG, "pool");
    std::lock_guard<std::mutex> lk(p->mu);
    PoolData *d = find_data(p, id);
    if (!d) return pool_fail(TLR_ERR_ARG, "unknown dataset " + std::to_string(id));
    if (n) *n = d->n;
    if (nb) *nb = d->nb;
    if (xy) *xy = d->xy;
    if (z) *z = d->z;
    if (perm) *perm = d->perm;
    if (last_max_rank) {
        int32_t m = 0;
        const int nt = (int)ceil_div(d->n, d->nb);
        if (d->hint.size() == (size_t)nt * nt)
            for (int i = 0; i < nt; ++i)
                for (int j = 0; j < i; ++j) m = std::max(m, d->hint[(size_t)i * nt + j]);
        *last_max_rank = m;
    }
    return TLR_OK;
}

int tlr_pool_submit(tlr_pool *p, int id, tlr_theta theta, double eps, int precision, int64_t *ticket) {
    if (!p || !ticket) return pool_fail(TLR_ERR_ARG, "pool/ticket");
    if (!args_ok(eps, precision)) return pool_fail(TLR_ERR_ARG, "eps/precision");
    std::lock_guard<std::mutex> lk(p->mu);
    PoolData *d = find_data(p, id);
    if (!d) return pool_fail(TLR_ERR_ARG, "unknown dataset " + std::to_string(id));
    return submit_locked(p, d, theta, eps, precision, ticket);
}

int tlr_pool_wait(tlr_pool *p, int64_t ticket, tlr_result *out, double *times_ms) {
    if (!p) return pool_fail(TLR_ERR_ARG, "pool");
    std::unique_lock<std::mutex> lk(p->mu);
    return wait_locked(p, lk, ticket, out, times_ms);
}

int tlr_pool_loglik(tlr_pool *p, int count, const int *ids, const tlr_theta *theta, double eps, int precision,
                    tlr_result *out, int *status) {
    if (!p || count < 0 || (count > 0 && (!ids || !theta))) return pool_fail(TLR_ERR_ARG, "pool/ids/theta");
    if (!args_ok(eps, precision)) return pool_fail(TLR_ERR_ARG, "eps/precision");
    std::unique_lock<std::mutex> lk(p->mu);
    for (int i = 0; i < count; ++i)
        if (!find_data(p, ids[i])) return pool_fail(TLR_ERR_ARG, "unknown dataset " + std::to_string(ids[i]));
    std::vector<int64_t> tickets((size_t)count);
    for (int i = 0; i < count; ++i)
        submit_locked(p, find_data(p, ids[i]), theta[i], eps, precision, &tickets[(size_t)i]);
    int first = TLR_OK;
    std::string first_err;
    for (int i = 0; i < count; ++i) {
        int st = wait_locked(p, lk, tickets[(size_t)i], out ? out + i : nullptr, nullptr);
        if (status) status[i] = st;
        if (st != TLR_OK && first == TLR_OK) {
            first = st;
            first_err = t_pool_err;
        }
    }
    if (first != TLR_OK) t_pool_err = first_err;
    return first;
}

int tlr_pool_mle(tlr_pool *p, int id, double eps, int precision, tlr_theta theta0, tlr_theta lo, tlr_theta hi,
                 double tol, int max_iter, tlr_theta *theta_hat, double *ll_hat, int *iters) {
    if (!p || !theta_hat || !ll_hat || !iters || max_iter <= 0 || !(tol > 0))
        return pool_fail(TLR_ERR_ARG, "mle outputs");
    if (!mle_bounds_ok(lo, hi)) return pool_fail(TLR_ERR_ARG, "bounds");
    if (!args_ok(eps, precision)) return pool_fail(TLR_ERR_ARG, "eps/precision");
    try {
        auto negll = [&](tlr_theta th) -> double {
            int64_t t = 0;
            int rc = tlr_pool_submit(p, id, th, eps, precision, &t);
            if (rc != TLR_OK) throw Error{rc, t_pool_err};
            tlr_result r;
            rc = tlr_pool_wait(p, t, &r, nullptr);
            if (rc == TLR_ERR_NOT_SPD || rc == TLR_ERR_RANK || rc == TLR_ERR_NAN) return INFINITY;
            if (rc != TLR_OK) throw Error{rc, t_pool_err};
            return -r.loglik;
        };
        mle_nelder_mead(negll, theta0, lo, hi, tol, max_iter, theta_hat, ll_hat, iters);
    } catch (const Error &e) {
        return pool_fail(e.code, e.msg);
    }
    return TLR_OK;
}

int tlr_pool_tune(tlr_pool *p, int id, tlr_theta theta, double eps, int precision, const int32_t *cands,
                  int ncand, int32_t *best, double *ms) {
    if (!p || !cands || ncand <= 0 || !best) return pool_fail(TLR_ERR_ARG, "pool/cands/best");
    if (!args_ok(eps, precision)) return pool_fail(TLR_ERR_ARG, "eps/precision");
    for (int c = 0; c < ncand; ++c)
        if (cands[c] < 16 || cands[c] > kMaxTile) return pool_fail(TLR_ERR_ARG, "candidate tile size");
    // Switches the idle dataset to tile size nb (dropping its factor storage
    // and rank map); false if that tile size cannot fit the budget.
    auto set_nb = [&](PoolData *d, int nb) -> bool {
        std::unique_lock<std::mutex> lk(p->mu);
        wait_idle(p, lk, d);
        const int maxrank = p->opts.maxrank > 0 ? std::min(p->opts.maxrank, nb) : nb / 2;
        const int64_t fb = factor_bytes(d->n, nb, maxrank, {}), wb = work_bytes(d->n, nb, maxrank, {});
        if (!p->adm.resize_check(id, fb, wb)) return false;
        p->adm.drop(id);
        tlr_mat *M = d->L;
        d->L = nullptr;
        d->nb = nb;
        d->maxrank = maxrank;
        d->hint.clear();
        d->pivot2 = 0.0;
        p->adm.resize(id, fb, wb);
        lk.unlock();
        if (M) {
            std::lock_guard<std::mutex> cl(p->ctl_mu);
            mat_free(M, p->ctl_stream);
            cudaStreamSynchronize(p->ctl_stream);
        }
        return true;
    };
    PoolData *d;
    int old_nb;
    {
        std::lock_guard<std::mutex> lk(p->mu);
        d = find_data(p, id);
        if (!d) return pool_fail(TLR_ERR_ARG, "unknown dataset " + std::to_string(id));
        old_nb = d->nb;
    }
    double best_ms = INFINITY;
    int best_nb = -1;
    for (int c = 0; c < ncand; ++c) {
        if (ms) ms[c] = -1.0;
        if (!set_nb(d, cands[c])) continue;
        tlr_result r{};
        for (int rep = 0; rep < 2; ++rep) {
            int64_t t = 0;
            int rc = tlr_pool_submit(p, id, theta, eps, precision, &t);
            if (rc == TLR_OK) rc = tlr_pool_wait(p, t, &r, nullptr);
            if (rc != TLR_OK) {
                std::string msg = t_pool_err;
                set_nb(d, old_nb);
                return pool_fail(rc, "tile size " + std::to_string(cands[c]) + ": " + msg);
            }
        }
        if (ms) ms[c] = r.ms_total;
        if (r.ms_total < best_ms) {
            best_ms = r.ms_total;
            best_nb = cands[c];
        }
    }
    if (best_nb < 0) {
        set_nb(d, old_nb);
        return pool_fail(TLR_ERR_OOM, "no candidate tile size fits the budget");
    }
    set_nb(d, best_nb);
    *best = best_nb;
    return TLR_OK;
}

int tlr_pool_configure(tlr_pool *p, int group, const tlr_buckets *b) {
    if (!p || group < 1 || group > kMaxGroup) return pool_fail(TLR_ERR_ARG, "pool/group (1..32)");
    const tlr_buckets v = b ? *b : default_buckets();
    if (!buckets_ok(v)) return pool_fail(TLR_ERR_ARG, "bucket sizes must be 1, 2, 4, 8 or 16, edges nondecreasing");
    std::lock_guard<std::mutex> lk(p->mu);
    p->cfg.group = group;
    p->cfg.buckets = v;
    return TLR_OK;
}

int tlr_pool_get_config(tlr_pool *p, int *group, tlr_buckets *b) {
    if (!p) return pool_fail(TLR_ERR_ARG, "pool");
    std::lock_guard<std::mutex> lk(p->mu);
    if (group) *group = p->cfg.group;
    if (b) *b = p->cfg.buckets;
    return TLR_OK;
}

int tlr_pool_autotune(tlr_pool *p, int count, const int *ids, const tlr_theta *theta, double eps, int precision,
                      int ncand, const int32_t *groups, const tlr_buckets *buckets, int rounds, double *evals_per_s,
                      int *best) {
    if (!p || count <= 0 || !ids || !theta || ncand <= 0 || !groups || rounds <= 0 || !best)
        return pool_fail(TLR_ERR_ARG, "autotune arguments");
    if (!args_ok(eps, precision)) return pool_fail(TLR_ERR_ARG, "eps/precision");
    for (int c = 0; c < ncand; ++c) {
        if (groups[c] < 1 || groups[c] > kMaxGroup) return pool_fail(TLR_ERR_ARG, "candidate group size");
        if (buckets && !buckets_ok(buckets[c])) return pool_fail(TLR_ERR_ARG, "candidate buckets");
    }
    int old_group;
    tlr_buckets old_b;
    tlr_pool_get_config(p, &old_group, &old_b);
    // every candidate starts from the same rank maps: one pass at the
    // current configuration first (it also sets the maps of new datasets)
    std::vector<tlr_result> out((size_t)count);
    std::vector<int> st((size_t)count);
    const int rc0 = tlr_pool_loglik(p, count, ids, theta, eps, precision, out.data(), st.data());
    if (rc0 == TLR_ERR_ARG) return rc0;  // unknown dataset (message already set)
    double best_rate = -1.0;
    int best_c = -1;
    for (int c = 0; c < ncand; ++c) {
        tlr_pool_configure(p, groups[c], buckets ? buckets + c : &old_b);
        const auto t0 = Clock::now();
        int ok = 0;
        for (int k = 0; k < rounds; ++k) {
            tlr_pool_loglik(p, count, ids, theta, eps, precision, out.data(), st.data());
            for (int q = 0; q < count; ++q) ok += st[(size_t)q] == TLR_OK;
        }
        const double sec = ms_between(t0, Clock::now()) / 1e3;
        const double rate = sec > 0 ? ok / sec : 0.0;
        if (evals_per_s) evals_per_s[c] = rate;
        if (rate > best_rate) {
            best_rate = rate;
            best_c = c;
        }
    }
    tlr_pool_configure(p, groups[best_c], buckets ? buckets + best_c : &old_b);
    *best = best_c;
    return TLR_OK;
}

int tlr_pool_footprint(int64_t n, int nb, int maxrank, int64_t *out) {
    if (!out || n <= 0 || nb < 16 || nb > kMaxTile || maxrank > nb) return pool_fail(TLR_ERR_ARG, "n/nb/maxrank/out");
    if (maxrank <= 0) maxrank = nb / 2;
    out[0] = n * 32;
    out[1] = factor_bytes(n, nb, maxrank, {});
    out[2] = work_bytes(n, nb, maxrank, {});
    return TLR_OK;
}

int tlr_pool_stats(tlr_pool *p, int64_t *out, int count) {
    if (!p || !out || count < 0) return pool_fail(TLR_ERR_ARG, "pool/out");
    std::lock_guard<std::mutex> lk(p->mu);
    int64_t fres = 0, nres = 0;
    for (auto &kv : p->data) {
        const Admission::Data &a = p->adm.data(kv.first);
        if (a.resident) {
            fres += a.fbytes;
            ++nres;
        }
    }
    const int64_t v[14] = {p->adm.budget(), p->adm.used(), p->adm.peak(), p->resident_bytes, fres, nres,
                           p->adm.evictions(), p->completed, (int64_t)p->adm.queued(), p->running,
                           p->max_running, p->allocations, p->groups, p->grouped};
    int k = std::min(count, 14);
    for (int i = 0; i < k; ++i) out[i] = v[i];
    return k;
}

int tlr_shard_place(int count, const int64_t *bytes, int nranks, const int64_t *budget, int32_t *rank_of) {
    if (count < 0 || nranks < 1 || (count > 0 && (!bytes || !rank_of))) return pool_fail(TLR_ERR_ARG, "shard arguments");
    for (int i = 0; i < count; ++i)
        if (bytes[i] < 0) return pool_fail(TLR_ERR_ARG, "negative footprint");
    std::vector<int> order((size_t)count);
    for (int i = 0; i < count; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return bytes[a] > bytes[b]; });
    std::vector<int64_t> load((size_t)nranks, 0);
    for (int i : order) {
        int best = -1;
        for (int r = 0; r < nranks; ++r) {
            if (budget && load[(size_t)r] + bytes[i] > budget[r]) continue;
            if (best < 0 || load[(size_t)r] < load[(size_t)best]) best = r;
        }
        if (best < 0) return pool_fail(TLR_ERR_OOM, "dataset " + std::to_string(i) + " fits no rank");
        load[(size_t)best] += bytes[i];
        rank_of[i] = best;
    }
    return TLR_OK;
}

int tlr_sched_simulate(int64_t budget, int workers, int ndata, const int64_t *base_bytes,
                       const int64_t *factor_bytes_, const int64_t *work_bytes_, int nreq, const int32_t *req_data,
                       const double *req_arrival, const double *req_cost, double *start, double *finish,
                       int64_t *peak_bytes, int64_t *evictions) {
    if (workers < 1 || ndata < 0 || nreq < 0 || (ndata > 0 && (!base_bytes || !factor_bytes_ || !work_bytes_)) ||
        (nreq > 0 && (!req_data || !req_arrival || !req_cost || !start || !finish)))
        return pool_fail(TLR_ERR_ARG, "simulate arguments");
    for (int i = 0; i < nreq; ++i)
        if (req_data[i] < 0 || req_data[i] >= ndata || !(req_cost[i] >= 0) ||
            (i > 0 && req_arrival[i] < req_arrival[i - 1]))
            return pool_fail(TLR_ERR_ARG, "requests");
    Admission adm(budget);
    for (int d = 0; d < ndata; ++d) {
        if (!adm.can_add(base_bytes[d], factor_bytes_[d], work_bytes_[d]))
            return pool_fail(TLR_ERR_OOM, "dataset " + std::to_string(d) + " does not fit");
        adm.add(base_bytes[d], factor_bytes_[d], work_bytes_[d]);
    }
    // running: (finish time, request)
    std::vector<std::pair<double, int>> run;
    int next = 0, done = 0;
    double now = 0.0;
    while (done < nreq) {
        // admit everything that can start now
        for (;;) {
            if ((int)run.size() >= workers) break;
            Admission::Req r{};
            bool alloc = false;
            if (!adm.admit(&r, &alloc, nullptr)) break;
            int q = (int)r.ticket;
            start[q] = now;
            finish[q] = now + req_cost[q];
            run.emplace_back(finish[q], q);
        }
        // next event: an arrival or a completion
        double t_arr = next < nreq ? req_arrival[next] : INFINITY;
        size_t first = 0;
        for (size_t k = 1; k < run.size(); ++k)
            if (run[k].first < run[first].first) first = k;
        double t_fin = run.empty() ? INFINITY : run[first].first;
        if (!std::isfinite(t_arr) && !std::isfinite(t_fin))
            return pool_fail(TLR_ERR_ARG, "simulation stalled");  // cannot happen: every dataset fits alone
        if (t_fin <= t_arr) {
            now = t_fin;
            adm.finish(req_data[run[first].second]);
            run.erase(run.begin() + (long)first);
            ++done;
        } else {
            now = t_arr;
            adm.enqueue(next, req_data[next]);
            ++next;
        }
    }
    if (peak_bytes) *peak_bytes = adm.peak();
    if (evictions) *evictions = adm.evictions();
    return TLR_OK;
}

}  // extern "C"
