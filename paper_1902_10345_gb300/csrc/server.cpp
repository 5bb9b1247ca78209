// Continuous-batching server for Jacobi solves.
//
// A worker thread owns the device work.  Each wave it (1) admits queued
// requests while the active set has free slots and the sum of footprints
// stays within the HBM budget, (2) advances every active grid by up to
// `quantum` steps in ONE persistent launch (grids stop early on their own
// tolerance inside the launch), (3) reads back the per-grid state, retires
// finished grids (copying the result into the caller's `out` when it sits in
// scratch) and frees their memory for the next admissions.  Requests that
// arrive while a wave runs are admitted at the next wave boundary, so their
// work overlaps on the device with the grids already running.
//
// A grid's pass schedule does not depend on the wave boundaries (waves end
// on multiples of the check stride, where passes end anyway), and its units,
// reduction order and termination test are those of a standalone solve, so
// every result is the same alone and in any mix.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

#include "launchset.h"

namespace sdfg {
int validate_grid(const void *in, const void *out, int R, int C, int ld, long long T, int dtype, const char *who);
int enqueue_persistent(LaunchSet &ls, DeviceState *st, cudaStream_t s);
}  // namespace sdfg

using namespace sdfg;

namespace {
enum ReqState { QUEUED = 0, ACTIVE = 1, DONE = 2 };

struct Request {
    uint64_t id = 0;
    sdfg_desc d{};
    int state = QUEUED;
    int status = SDFG_PENDING;
    int t = 0;           // steps completed
    int cur = 2;         // buffer holding the state
    double r_ref2 = 0.0;
    double rel = 0.0;
    int ld_int = 0;
    void *scratch = nullptr;
    void *stage_in = nullptr, *stage_out = nullptr;
    size_t footprint = 0;
    bool pause = false;  // snapshot requested
    CUtensorMap tm[3];   // encoded once at admission
};
}  // namespace

struct sdfg_server {
    size_t budget = 0;
    int max_slots = 0;
    int quantum = 0;
    int check_stride = 0;
    int device = 0;
    int dtype = -1;
    int seg_rows = 96;  // segment height of every grid's units
    bool k_fixed = false;  // k chosen by sdfg_server_set_config

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Request> reqs;
    std::vector<uint64_t> active;
    size_t used = 0;
    uint64_t next_id = 1;
    size_t unfinished = 0;
    bool stopping = false;
    int fatal = SDFG_OK;

    std::thread worker;
    cudaStream_t stream = nullptr;
    LaunchSet ls;
    PState *h_state = nullptr;  // pinned
    size_t h_state_cap = 0;
};

static size_t footprint_of(const sdfg_desc &d, int *ld_int, bool *staged) {
    const int S = dtype_bytes(d.dtype);
    *staged = !(tma_compatible(d.in, d.ld, d.dtype) && tma_compatible(d.out, d.ld, d.dtype));
    *ld_int = *staged ? (d.cols + 31) / 32 * 32 : d.ld;
    const size_t grid = static_cast<size_t>(d.rows) * (*ld_int) * S;
    // caller's in and out + the scratch grid (+ two staging grids)
    return static_cast<size_t>(d.rows) * d.ld * S * 2 + grid * (*staged ? 3 : 1);
}

static void release_request(sdfg_server *sv, Request &r) {
    for (void *p : {r.scratch, r.stage_in, r.stage_out})
        if (p) cudaFreeAsync(p, sv->stream);
    r.scratch = r.stage_in = r.stage_out = nullptr;
    sv->used -= r.footprint;
    r.footprint = 0;
}

static void finish_request(sdfg_server *sv, Request &r, int status) {
    r.state = DONE;
    r.status = status;
    --sv->unfinished;
}

// Admit queued requests (lock held).  Allocation failures fail the request.
static void admit_locked(sdfg_server *sv) {
    while (!sv->queue.empty() && static_cast<int>(sv->active.size()) < sv->max_slots) {
        Request &r = sv->reqs[sv->queue.front()];
        bool staged = false;
        const size_t fp = footprint_of(r.d, &r.ld_int, &staged);
        if (sv->used + fp > sv->budget && !sv->active.empty()) break;  // wait for memory
        sv->queue.pop_front();
        const int S = dtype_bytes(r.d.dtype);
        const size_t bytes = static_cast<size_t>(r.d.rows) * r.ld_int * S;
        int rc = scratch_alloc(&r.scratch, bytes, sv->stream);
        if (rc == SDFG_OK && staged) {
            rc = scratch_alloc(&r.stage_in, bytes, sv->stream);
            if (rc == SDFG_OK) rc = scratch_alloc(&r.stage_out, bytes, sv->stream);
            if (rc == SDFG_OK && cudaMemcpy2DAsync(r.stage_in, static_cast<size_t>(r.ld_int) * S, r.d.in,
                                                   static_cast<size_t>(r.d.ld) * S, static_cast<size_t>(r.d.cols) * S,
                                                   r.d.rows, cudaMemcpyDeviceToDevice, sv->stream) != cudaSuccess)
                rc = SDFG_ERR_CUDA;
        }
        r.footprint = fp;
        sv->used += fp;
        if (rc != SDFG_OK) {
            release_request(sv, r);
            finish_request(sv, r, rc);
            continue;
        }
        r.state = ACTIVE;
        r.t = r.d.t_start;
        r.r_ref2 = r.d.r_first2;
        r.cur = (r.d.in == r.d.out && !staged) ? 0 : 2;
        {
            const void *bufs[3] = {r.stage_out ? r.stage_out : r.d.out, r.scratch,
                                   r.stage_in ? r.stage_in : r.d.in};
            const int W = 32 * lane_cols(dtype_bytes(r.d.dtype));
            for (int b = 0; b < 3 && rc == SDFG_OK; ++b)
                rc = encode_tmap(&r.tm[b], bufs[b], r.d.dtype, r.d.rows, r.d.cols, r.ld_int, W);
        }
        if (rc != SDFG_OK) {
            release_request(sv, r);
            finish_request(sv, r, rc);
            continue;
        }
        sv->active.push_back(r.id);
    }
}

static int copy_result(sdfg_server *sv, Request &r, int final_buf) {
    const int S = dtype_bytes(r.d.dtype);
    const void *src = final_buf == 0 ? (r.stage_out ? r.stage_out : r.d.out)
                                     : (final_buf == 1 ? r.scratch : (r.stage_in ? r.stage_in : r.d.in));
    if (src == r.d.out) return SDFG_OK;
    cudaError_t e = cudaMemcpy2DAsync(r.d.out, static_cast<size_t>(r.d.ld) * S, src, static_cast<size_t>(r.ld_int) * S,
                                      static_cast<size_t>(r.d.cols) * S, r.d.rows, cudaMemcpyDeviceToDevice,
                                      sv->stream);
    return e == cudaSuccess ? SDFG_OK : cuda_error(e, "server result copy");
}

static void worker_main(sdfg_server *sv) {
    cudaSetDevice(sv->device);
    DeviceState *st = nullptr;
    if (current_device(&st) != SDFG_OK) {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->fatal = SDFG_ERR_UNSUPPORTED;
        for (auto &kv : sv->reqs)
            if (kv.second.state != DONE) finish_request(sv, kv.second, SDFG_ERR_UNSUPPORTED);
        sv->cv_done.notify_all();
        return;
    }
    std::vector<GridRun> runs;
    std::vector<uint64_t> ids;
    while (true) {
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            admit_locked(sv);
            sv->cv_done.notify_all();  // failed admissions
            while (sv->active.empty() && !sv->stopping) {
                sv->cv_work.wait(lk);
                admit_locked(sv);
                sv->cv_done.notify_all();
            }
            if (sv->active.empty() && sv->stopping) break;
            // one wave over the active set
            runs.clear();
            ids = sv->active;
            for (uint64_t id : ids) {
                Request &r = sv->reqs[id];
                GridRun g;
                g.buf[0] = r.stage_out ? r.stage_out : r.d.out;
                g.buf[1] = r.scratch;
                g.buf[2] = r.cur == 2 ? (r.stage_in ? r.stage_in : const_cast<void *>(r.d.in)) : nullptr;
                g.ld = r.ld_int;
                g.R = r.d.rows;
                g.C = r.d.cols;
                g.t0 = r.t;
                g.T_cap = r.d.T;
                g.steps = std::min(sv->quantum, r.d.T - r.t);
                g.cur = r.cur;
                g.tol = r.d.tol;
                g.r_ref2 = r.r_ref2;
                g.seg_rows = sv->seg_rows;
                g.tmaps = r.tm;
                runs.push_back(g);
            }
        }
        int rc = sv->ls.build(runs);
        if (rc == SDFG_OK) rc = sv->ls.upload(sv->stream);
        if (rc == SDFG_OK) rc = enqueue_persistent(sv->ls, st, sv->stream);
        const size_t n = runs.size();
        if (rc == SDFG_OK && sv->h_state_cap < n) {
            if (sv->h_state) cudaFreeHost(sv->h_state);
            sv->h_state = nullptr;
            sv->h_state_cap = 0;
            if (cudaMallocHost(&sv->h_state, n * sizeof(PState)) != cudaSuccess)
                rc = SDFG_ERR_NOMEM;
            else
                sv->h_state_cap = n;
        }
        if (rc == SDFG_OK && n)
            if (cudaMemcpyAsync(sv->h_state, sv->ls.L.state, n * sizeof(PState), cudaMemcpyDeviceToHost,
                                sv->stream) != cudaSuccess)
                rc = SDFG_ERR_CUDA;
        int errw = 0;
        if (rc == SDFG_OK && cudaStreamSynchronize(sv->stream) != cudaSuccess) rc = SDFG_ERR_CUDA;
        if (rc == SDFG_OK && cudaMemcpy(&errw, st->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = SDFG_ERR_CUDA;
        if (rc == SDFG_OK && errw) {
            cudaMemset(st->d_err, 0, sizeof(int));
            rc = SDFG_ERR_TIMEOUT;
        }
        std::lock_guard<std::mutex> lk(sv->mu);
        std::vector<uint64_t> still;
        for (size_t g = 0; g < n; ++g) {
            Request &r = sv->reqs[ids[g]];
            if (rc != SDFG_OK) {
                release_request(sv, r);
                finish_request(sv, r, rc);
                continue;
            }
            const PState &S = sv->h_state[g];
            const bool tol_mode = r.d.tol > 0.0;
            bool done = false;
            int final_buf = 0;
            if (tol_mode) {
                r.r_ref2 = S.r_ref2;
                r.rel = S.rel;
                if (S.stop_pass >= 0) {
                    done = true;
                    r.t = S.steps_done;
                    final_buf = S.final_buf;
                } else {
                    r.t += runs[g].steps;
                    r.cur = sv->ls.last_dst[g];
                }
            } else {
                r.t += runs[g].steps;
                r.cur = sv->ls.last_dst[g];
                if (r.t >= r.d.T) {
                    done = true;
                    final_buf = r.cur;
                }
            }
            if (done) {
                const int crc = copy_result(sv, r, final_buf);
                release_request(sv, r);
                r.d.steps_done = r.t;
                r.d.rel_residual = tol_mode ? r.rel : 0.0;
                r.d.r_first2 = r.r_ref2;
                finish_request(sv, r, crc);
            } else if (r.pause) {
                // snapshot: the grid after r.t steps goes to `out`
                const int crc = copy_result(sv, r, r.cur);
                release_request(sv, r);
                r.d.steps_done = r.t;
                r.d.rel_residual = tol_mode ? r.rel : 0.0;
                r.d.r_first2 = r.r_ref2;
                finish_request(sv, r, crc == SDFG_OK ? SDFG_PAUSED : crc);
            } else {
                still.push_back(r.id);
            }
        }
        sv->active.swap(still);
        // results copied to `out` must be complete before poll reports them
        cudaStreamSynchronize(sv->stream);
        sv->cv_done.notify_all();
    }
}

extern "C" int sdfg_server_create(sdfg_server **server, size_t hbm_budget_bytes, int max_slots, int quantum_steps,
                                  int check_stride, int device) {
    if (!server || hbm_budget_bytes == 0 || max_slots < 1 || quantum_steps < 1 || check_stride < 1 ||
        quantum_steps % check_stride != 0)
        return set_error(SDFG_ERR_INVAL,
                         "sdfg_server_create: need budget > 0, max_slots >= 1, check_stride >= 1 and quantum_steps a "
                         "positive multiple of check_stride");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return set_error(SDFG_ERR_INVAL, "sdfg_server_create: bad device %d", device);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    DeviceState *st = nullptr;
    int rc = current_device(&st);
    sdfg_server *sv = nullptr;
    if (rc == SDFG_OK) {
        sv = new sdfg_server();
        sv->budget = hbm_budget_bytes;
        sv->max_slots = max_slots;
        sv->quantum = quantum_steps;
        sv->check_stride = check_stride;
        sv->device = device;
        sv->ls.check_stride = check_stride;
        sv->ls.warps = 4;
        e = cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) rc = cuda_error(e, "server stream");
    }
    cudaSetDevice(prev);
    if (rc != SDFG_OK) {
        delete sv;
        return rc;
    }
    sv->worker = std::thread(worker_main, sv);
    *server = sv;
    return SDFG_OK;
}

extern "C" int sdfg_server_set_config(sdfg_server *sv, const sdfg_config *cfg) {
    if (!sv || !cfg) return set_error(SDFG_ERR_INVAL, "sdfg_server_set_config: null argument");
    if ((cfg->k != 0 && !depth_supported(cfg->k)) || cfg->seg_rows < 0 || cfg->warps < 0 || cfg->warps > 4)
        return set_error(SDFG_ERR_INVAL, "sdfg_server_set_config: k must be 1, 2, 4 or 8; warps 0..4");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (!sv->active.empty() || !sv->queue.empty())
        return set_error(SDFG_ERR_BUSY, "sdfg_server_set_config: requests are in flight");
    if (cfg->k) sv->ls.k = cfg->k;
    if (cfg->seg_rows) sv->seg_rows = cfg->seg_rows;
    if (cfg->warps) sv->ls.warps = cfg->warps;
    sv->k_fixed = cfg->k != 0;
    return SDFG_OK;
}

extern "C" int sdfg_server_submit(sdfg_server *sv, const sdfg_desc *desc, uint64_t *req_id) {
    if (!sv || !desc || !req_id) return set_error(SDFG_ERR_INVAL, "sdfg_server_submit: null argument");
    const sdfg_desc &d = *desc;
    int rc = validate_grid(d.in, d.out, d.rows, d.cols, d.ld, d.T, d.dtype, "sdfg_server_submit");
    if (rc != SDFG_OK) return rc;
    if (!(d.tol >= 0.0)) return set_error(SDFG_ERR_INVAL, "sdfg_server_submit: tol must be >= 0");
    if (d.t_start < 0 || d.t_start > d.T || !(d.r_first2 >= 0.0))
        return set_error(SDFG_ERR_INVAL, "sdfg_server_submit: need 0 <= t_start <= T and r_first2 >= 0");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stopping) return set_error(SDFG_ERR_BUSY, "sdfg_server_submit: server is shutting down");
    if (sv->fatal != SDFG_OK) return set_error(sv->fatal, "sdfg_server_submit: server failed to start");
    if (sv->dtype >= 0 && d.dtype != sv->dtype)
        return set_error(SDFG_ERR_INVAL, "sdfg_server_submit: a server serves one dtype");
    int ld_int;
    bool staged;
    const size_t fp = footprint_of(d, &ld_int, &staged);
    if (fp > sv->budget) return set_error(SDFG_ERR_NOMEM, "sdfg_server_submit: request needs %zu bytes > budget", fp);
    sv->dtype = d.dtype;
    sv->ls.dtype = d.dtype;
    // serving mixes many small grids: the 4-column halo of k = 4 wastes less
    // of each 128-column strip than k = 8 (measured on the served workload)
    if (!sv->k_fixed) sv->ls.k = d.dtype == SDFG_F64 ? default_depth(d.dtype) : 4;
    Request r;
    r.id = sv->next_id++;
    r.d = d;
    r.d.status = SDFG_PENDING;
    ++sv->unfinished;
    if (d.rows < 3 || d.cols < 3 || d.T == d.t_start) {
        // nothing to iterate: a copy, done at once
        const int S = dtype_bytes(d.dtype);
        if (d.rows > 0 && d.cols > 0 && d.in != d.out) {
            cudaMemcpy2DAsync(d.out, static_cast<size_t>(d.ld) * S, d.in, static_cast<size_t>(d.ld) * S,
                              static_cast<size_t>(d.cols) * S, d.rows, cudaMemcpyDeviceToDevice, sv->stream);
            cudaStreamSynchronize(sv->stream);
        }
        r.d.steps_done = (d.rows < 3 || d.cols < 3) ? d.T : d.t_start;
        r.d.rel_residual = 0.0;
        r.d.r_first2 = d.r_first2;
        finish_request(sv, r, SDFG_OK);
        sv->reqs[r.id] = r;
        sv->cv_done.notify_all();
    } else {
        sv->reqs[r.id] = r;
        // higher priority first, FIFO within a priority
        auto it = sv->queue.end();
        while (it != sv->queue.begin() && sv->reqs[*(it - 1)].d.priority < d.priority) --it;
        sv->queue.insert(it, r.id);
        sv->cv_work.notify_one();
    }
    *req_id = r.id;
    return SDFG_OK;
}

extern "C" int sdfg_server_poll(sdfg_server *sv, uint64_t req_id, sdfg_desc *result) {
    if (!sv) return set_error(SDFG_ERR_INVAL, "sdfg_server_poll: null server");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(req_id);
    if (it == sv->reqs.end()) return set_error(SDFG_ERR_INVAL, "sdfg_server_poll: unknown request %llu",
                                               static_cast<unsigned long long>(req_id));
    Request &r = it->second;
    if (r.state != DONE) return SDFG_PENDING;  // (a paused request is DONE with status SDFG_PAUSED)
    const int status = r.status;
    if (result) {
        *result = r.d;
        result->status = status;
    }
    sv->reqs.erase(it);
    return status;
}

extern "C" int sdfg_server_snapshot(sdfg_server *sv, uint64_t req_id) {
    if (!sv) return set_error(SDFG_ERR_INVAL, "sdfg_server_snapshot: null server");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(req_id);
    if (it == sv->reqs.end() || it->second.state == DONE)
        return set_error(SDFG_ERR_INVAL, "sdfg_server_snapshot: request %llu is unknown or finished",
                         static_cast<unsigned long long>(req_id));
    Request &r = it->second;
    if (r.state == QUEUED) {
        // never started: its state is its input
        for (auto q = sv->queue.begin(); q != sv->queue.end(); ++q)
            if (*q == req_id) {
                sv->queue.erase(q);
                break;
            }
        const int S = dtype_bytes(r.d.dtype);
        if (r.d.in != r.d.out) {
            cudaMemcpy2DAsync(r.d.out, static_cast<size_t>(r.d.ld) * S, r.d.in, static_cast<size_t>(r.d.ld) * S,
                              static_cast<size_t>(r.d.cols) * S, r.d.rows, cudaMemcpyDeviceToDevice, sv->stream);
            cudaStreamSynchronize(sv->stream);
        }
        r.d.steps_done = r.d.t_start;
        finish_request(sv, r, SDFG_PAUSED);
        sv->cv_done.notify_all();
        return SDFG_OK;
    }
    r.pause = true;
    return SDFG_OK;
}

extern "C" int sdfg_server_drain(sdfg_server *sv, int timeout_ms) {
    if (!sv) return set_error(SDFG_ERR_INVAL, "sdfg_server_drain: null server");
    std::unique_lock<std::mutex> lk(sv->mu);
    const auto pred = [&] { return sv->unfinished == 0; };
    if (timeout_ms < 0) {
        sv->cv_done.wait(lk, pred);
        return SDFG_OK;
    }
    if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
        return set_error(SDFG_ERR_TIMEOUT, "sdfg_server_drain: %zu requests still running after %d ms",
                         sv->unfinished, timeout_ms);
    return SDFG_OK;
}

extern "C" int sdfg_server_destroy(sdfg_server *sv) {
    if (!sv) return SDFG_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
        // queued requests that never started are cancelled
        for (uint64_t id : sv->queue) {
            Request &r = sv->reqs[id];
            finish_request(sv, r, SDFG_ERR_BUSY);
        }
        sv->queue.clear();
        sv->cv_work.notify_all();
    }
    if (sv->worker.joinable()) sv->worker.join();
    cudaSetDevice(sv->device);
    sv->ls.release(sv->stream);
    if (sv->stream) {
        cudaStreamSynchronize(sv->stream);
        cudaStreamDestroy(sv->stream);
    }
    if (sv->h_state) cudaFreeHost(sv->h_state);
    delete sv;
    return SDFG_OK;
}
