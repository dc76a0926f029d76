// server.cpp - solve server: continuous batching of independent solves, each
// with its own mesh, over the library's own entry points (vie_set_mesh,
// vie_solve).  A deployment layer; the paper solves one configuration at a
// time.
//
// Slots: n host threads, each with its own context (device mesh, Z, block
// inverses of Eq. (6), Krylov state) and its own non-blocking CUDA stream, so
// the kernels of different slots overlap on the GPU.  Admission: a queued
// request goes to a free slot once its device footprint fits in the HBM
// budget beside what the other slots hold; requests are taken in arrival
// order, and a later request that fits may pass the head of the queue (at
// most MAX_PASSED times per waiting request).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/vie.h"
#include "vie_internal.h"

namespace vie {
size_t gj_pack_bytes(int n);   // packing scratch of the block inversion (linalg.cu)
}

namespace {

using clk = std::chrono::steady_clock;
constexpr int MAX_PASSED = 8;

struct Job {
    uint64_t ticket = 0;
    std::vector<double> verts;
    std::vector<int32_t> tets, dom;
    vie_mesh mesh{};
    vie_request req{};
    size_t footprint = 0;
    int passed = 0;          // times a later request was admitted before this one
    bool done = false;
    std::atomic<int> cancel{0};   // set by vie_server_cancel while the request runs
    vie_result res{};
    clk::time_point t_submit, t_start, t_end;
};

// Device bytes one slot holds for a mesh (upper bound): N is bounded by the
// number of distinct faces; the block inverses of Eq. (6) by one N x N matrix;
// the near-image masks by the tetrahedron and boundary/interface face counts.
size_t mesh_footprint(const vie_mesh &m, const vie_options &opt) {
    struct Key {
        int32_t v[3];
        bool operator==(const Key &o) const { return v[0] == o.v[0] && v[1] == o.v[1] && v[2] == o.v[2]; }
    };
    struct Hash {
        size_t operator()(const Key &k) const {
            return ((size_t)(uint32_t)k.v[0] * 73856093u) ^ ((size_t)(uint32_t)k.v[1] * 19349663u) ^
                   ((size_t)(uint32_t)k.v[2] * 83492791u);
        }
    };
    std::unordered_map<Key, std::array<int32_t, 2>, Hash> faces;
    faces.reserve((size_t)m.n_tets * 3);
    for (int32_t t = 0; t < m.n_tets; ++t)
        for (int i = 0; i < 4; ++i) {
            Key k;
            int c = 0;
            for (int j = 0; j < 4; ++j)
                if (j != i) k.v[c++] = m.tets[4 * (size_t)t + j];
            std::sort(k.v, k.v + 3);
            auto it = faces.find(k);
            if (it == faces.end()) faces.emplace(k, std::array<int32_t, 2>{t, -1});
            else it->second[1] = t;
        }
    size_t n_faces = faces.size(), n_bnd = 0, n_jump = 0;
    for (auto &f : faces) {
        if (f.second[1] < 0) ++n_bnd;
        else if (m.tet_domain[f.second[0]] != m.tet_domain[f.second[1]]) ++n_jump;
    }
    const size_t N = n_faces, ld = (N + 3) / 4 * 4, nt = (size_t)m.n_tets;
    const size_t nf = n_bnd + n_jump, nh = n_bnd;
    const size_t sz = opt.precision == VIE_FP64 ? 8 : 4;
    const size_t mres = (size_t)std::max(2, opt.restart);
    size_t b = 2 * sz * ld * N;                          // Z
    const size_t l16 = (N + 127) / 128 * 128;            // row stride of the 16-bit (interleaved) copies
    if (opt.precision == VIE_FP16 || opt.precision == VIE_BF16) b += 2 * 2 * l16 * N;   // its 16-bit copy
    b += 8 * ld * N + 4 * l16 * N;                       // block inverses (FP32 and FP16), bounded by N^2
    b += 2 * vie::gj_pack_bytes((int)N);                 // packing scratch of the inversion (two blocks at once)
    b += sz * 4 * N * (mres + 3) + 8 * 4 * N * 4;        // Krylov basis and vectors, x, r, b, coefficients
    b += 2 * (nt * nt + nt * nf + nh * nt + nh * nf);    // near-image masks
    b += nt * 4096 + ((size_t)64 << 20);                 // per-element arrays, lists, tables, small buffers
    return b;
}

}  // namespace

struct vie_server {
    int device = 0;
    vie_options opt{};
    size_t budget = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Job>> jobs;
    std::vector<std::thread> workers;
    std::vector<size_t> held;   // bytes each slot holds or has reserved
    size_t reserved = 0, peak_reserved = 0;
    uint64_t next_ticket = 1;
    int64_t submitted = 0, completed = 0, rejected = 0, running = 0, max_running = 0, cancelled = 0;
    bool stop = false;

    // index in the queue of the request slot k may take now, or -1
    int pick(int k) {
        for (size_t i = 0; i < queue.size(); ++i) {
            const Job *j = queue[i];
            const size_t after = reserved - held[k] + std::max(held[k], j->footprint);
            if (after <= budget) return (int)i;
            // the head (and any earlier request) is waiting: a later one may pass
            // it only a bounded number of times
            if (j->passed >= MAX_PASSED) return -1;
        }
        return -1;
    }

    void work(int k) {
        cudaSetDevice(device);
        vie_ctx *ctx = nullptr;
        cudaStream_t st = nullptr;
        int init = vie_create(&ctx, device, &opt);
        if (init == VIE_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) init = VIE_ECUDA;
        for (;;) {
            Job *j = nullptr;
            {
                std::unique_lock<std::mutex> lock(mu);
                int idx = -1;
                for (;;) {
                    if (stop) break;
                    if ((idx = pick(k)) >= 0) break;
                    if (!queue.empty() && held[k] > 0) {
                        // idle with requests waiting for memory: give this slot's back
                        vie::release_device_memory(ctx);
                        reserved -= held[k];
                        held[k] = 0;
                        cv_work.notify_all();
                        continue;
                    }
                    cv_work.wait(lock);
                }
                if (stop) break;
                j = queue[idx];
                for (int i = 0; i < idx; ++i) queue[i]->passed++;
                queue.erase(queue.begin() + idx);
                // a slot holding much more than the request needs gives the rest back
                if (held[k] > 2 * j->footprint) {
                    vie::release_device_memory(ctx);
                    reserved -= held[k];
                    held[k] = 0;
                }
                const size_t now = std::max(held[k], j->footprint);
                reserved += now - held[k];
                held[k] = now;
                peak_reserved = std::max(peak_reserved, reserved);
                running++;
                max_running = std::max(max_running, running);
                j->t_start = clk::now();
            }
            vie_result res{};
            int rc = init;
            if (rc == VIE_OK)
                rc = vie_set_mesh(ctx, j->mesh.verts, j->mesh.n_verts, j->mesh.tets, j->mesh.n_tets,
                                  j->mesh.tet_domain, j->mesh.n_domains, j->mesh.period_a, j->mesh.period_b,
                                  j->mesh.active_domain);
            if (rc == VIE_OK) {
                vie::set_cancel_flag(ctx, &j->cancel);
                rc = vie_solve(ctx, &j->req, &res, st);
                vie::set_cancel_flag(ctx, nullptr);
            }
            res.status = rc;
            {
                std::lock_guard<std::mutex> lock(mu);
                j->t_end = clk::now();
                auto ms = [](clk::time_point a, clk::time_point b) {
                    return std::chrono::duration<double, std::milli>(b - a).count();
                };
                res.t_queue_ms = ms(j->t_submit, j->t_start);
                res.t_latency_ms = ms(j->t_submit, j->t_end);
                j->res = res;
                j->done = true;
                // the request's inputs are no longer needed
                std::vector<double>().swap(j->verts);
                std::vector<int32_t>().swap(j->tets);
                std::vector<int32_t>().swap(j->dom);
                running--;
                completed++;
                if (rc == VIE_CANCELLED) cancelled++;
            }
            cv_done.notify_all();
            cv_work.notify_all();   // memory may have been released for a waiting request
        }
        if (st) cudaStreamDestroy(st);
        vie_destroy(ctx);
    }
};

extern "C" {

int vie_server_create(vie_server **out, int device, const vie_options *opt, int32_t n_slots,
                      int64_t hbm_budget_bytes) {
    if (!out || n_slots < 1 || n_slots > 64 || hbm_budget_bytes < 0) return VIE_EINVAL;
    *out = nullptr;
    int nd = 0;
    if (cudaGetDeviceCount(&nd) != cudaSuccess || device < 0 || device >= nd) return VIE_ECUDA;
    if (cudaSetDevice(device) != cudaSuccess) return VIE_ECUDA;
    vie_server *s = new (std::nothrow) vie_server();
    if (!s) return VIE_ENOMEM;
    s->device = device;
    vie_default_options(&s->opt);
    if (opt) s->opt = *opt;
    if (hbm_budget_bytes > 0) {
        s->budget = (size_t)hbm_budget_bytes;
    } else {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { delete s; return VIE_ECUDA; }
        const size_t headroom = total_b / 20 + ((size_t)1 << 30);
        s->budget = free_b > headroom ? free_b - headroom : 0;
    }
    s->held.assign(n_slots, 0);
    for (int k = 0; k < n_slots; ++k) s->workers.emplace_back([s, k] { s->work(k); });
    *out = s;
    return VIE_OK;
}

int vie_server_submit(vie_server *s, const vie_mesh *mesh, const vie_request *req, uint64_t *ticket,
                      int64_t *footprint_bytes) {
    if (!s || !mesh || !req || !ticket) return VIE_EINVAL;
    if (!mesh->verts || !mesh->tets || !mesh->tet_domain || mesh->n_verts < 4 || mesh->n_tets < 1) return VIE_EINVAL;
    for (int64_t i = 0; i < 4 * (int64_t)mesh->n_tets; ++i)
        if (mesh->tets[i] < 0 || mesh->tets[i] >= mesh->n_verts) return VIE_EINVAL;
    std::unique_ptr<Job> j(new (std::nothrow) Job());
    if (!j) return VIE_ENOMEM;
    j->verts.assign(mesh->verts, mesh->verts + 3 * (size_t)mesh->n_verts);
    j->tets.assign(mesh->tets, mesh->tets + 4 * (size_t)mesh->n_tets);
    j->dom.assign(mesh->tet_domain, mesh->tet_domain + (size_t)mesh->n_tets);
    j->mesh = *mesh;
    j->mesh.verts = j->verts.data();
    j->mesh.tets = j->tets.data();
    j->mesh.tet_domain = j->dom.data();
    j->req = *req;
    j->footprint = mesh_footprint(j->mesh, s->opt);
    if (footprint_bytes) *footprint_bytes = (int64_t)j->footprint;
    std::lock_guard<std::mutex> lock(s->mu);
    if (j->footprint > s->budget) {
        s->rejected++;
        return VIE_ENOMEM;
    }
    j->ticket = s->next_ticket++;
    j->t_submit = clk::now();
    *ticket = j->ticket;
    s->queue.push_back(j.get());
    s->jobs.emplace(j->ticket, std::move(j));
    s->submitted++;
    s->cv_work.notify_all();
    return VIE_OK;
}

int vie_server_poll(vie_server *s, uint64_t ticket, vie_result *res, int32_t wait_ms) {
    if (!s || !res) return VIE_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return VIE_EINVAL;
    Job *j = it->second.get();
    if (!j->done && wait_ms != 0) {
        if (wait_ms < 0) s->cv_done.wait(lock, [&] { return j->done; });
        else s->cv_done.wait_for(lock, std::chrono::milliseconds(wait_ms), [&] { return j->done; });
    }
    if (!j->done) return VIE_PENDING;
    *res = j->res;
    s->jobs.erase(it);
    return VIE_OK;
}

int vie_server_cancel(vie_server *s, uint64_t ticket) {
    if (!s) return VIE_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return VIE_EINVAL;
    Job *j = it->second.get();
    if (j->done) return VIE_OK;   // finished first: it keeps its result
    auto q = std::find(s->queue.begin(), s->queue.end(), j);
    if (q != s->queue.end()) {    // still queued: never runs
        s->queue.erase(q);
        j->t_start = j->t_end = clk::now();
        j->res = vie_result{};
        j->res.status = VIE_CANCELLED;
        j->res.t_latency_ms = std::chrono::duration<double, std::milli>(j->t_end - j->t_submit).count();
        j->done = true;
        s->cancelled++;
        s->cv_done.notify_all();
        s->cv_work.notify_all();
        return VIE_OK;
    }
    j->cancel.store(1);           // running: the solve stops at its next check
    return VIE_OK;
}

int vie_server_get_stats(vie_server *s, vie_server_stats *out) {
    if (!s || !out) return VIE_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->queued = (int64_t)s->queue.size();
    out->running = s->running;
    out->max_running = s->max_running;
    out->budget_bytes = (int64_t)s->budget;
    out->reserved_bytes = (int64_t)s->reserved;
    out->peak_reserved_bytes = (int64_t)s->peak_reserved;
    out->cancelled = s->cancelled;
    return VIE_OK;
}

void vie_server_destroy(vie_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->queue.clear();
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    delete s;
}

}  // extern "C"
