// Serving loop: many concurrent jobs (each a batch of environments with its
// own bodies, cameras and state) send step+render requests; the server keeps
// every admitted job resident on the device, admits waiting jobs as the HBM
// budget frees up, and batches the requests pending at each moment into one
// work-list launch per phase.  Iterations are pipelined like the paper's
// data-generation loop (Sec. 3.1): the sim launch of iteration k+1 runs on
// the sim stream while iteration k renders on the render stream, so requests
// that arrive while others are on the GPU join the next launch (continuous
// batching) and their work overlaps on the device.
//
// A job's results do not depend on the mix: every environment is stepped and
// rendered by the same kernel code from its own state, and its pose slots
// and frame belong to it.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "env.cuh"

using namespace vuda;

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// Host copy of a job's scene, kept until the job is admitted.
struct SceneCopy {
    std::vector<int32_t> body_off, mesh_id, mesh_vert_off, mesh_tri_off, mesh_tris, cam_off, cam_w, cam_h;
    std::vector<float> pos, quat, vel, ang, dims, im, ii, scale, verts, eye, right, up, fwd, fpy;
    std::vector<uint8_t> type;
    std::vector<uint32_t> albedo;
    vuda_scene view{};

    explicit SceneCopy(const vuda_scene& s) {
        const int E = s.num_envs, B = E ? s.body_off[E] : 0, C = E ? s.cam_off[E] : 0, M = s.num_meshes;
        auto cp = [](auto& v, const auto* p, size_t n) { v.assign(p, p + n); };
        cp(body_off, s.body_off, E + 1);
        cp(pos, s.pos, 3 * (size_t)B);
        cp(quat, s.quat, 4 * (size_t)B);
        cp(vel, s.vel, 3 * (size_t)B);
        cp(ang, s.angvel, 3 * (size_t)B);
        cp(type, s.shape_type, B);
        cp(dims, s.shape_dims, 3 * (size_t)B);
        cp(im, s.inv_mass, B);
        cp(ii, s.inv_inertia, 3 * (size_t)B);
        cp(mesh_id, s.mesh_id, B);
        cp(scale, s.mesh_scale, 3 * (size_t)B);
        cp(albedo, s.albedo, B);
        cp(mesh_vert_off, s.mesh_vert_off, M + 1);
        cp(mesh_tri_off, s.mesh_tri_off, M + 1);
        cp(verts, s.mesh_verts, 3 * (size_t)s.mesh_vert_off[M]);
        cp(mesh_tris, s.mesh_tris, 3 * (size_t)s.mesh_tri_off[M]);
        cp(cam_off, s.cam_off, E + 1);
        cp(cam_w, s.cam_w, C);
        cp(cam_h, s.cam_h, C);
        cp(eye, s.cam_eye, 3 * (size_t)C);
        cp(right, s.cam_right, 3 * (size_t)C);
        cp(up, s.cam_up, 3 * (size_t)C);
        cp(fwd, s.cam_fwd, 3 * (size_t)C);
        cp(fpy, s.cam_fpy, C);
        view = s;
        view.body_off = body_off.data();
        view.pos = pos.data();
        view.quat = quat.data();
        view.vel = vel.data();
        view.angvel = ang.data();
        view.shape_type = type.data();
        view.shape_dims = dims.data();
        view.inv_mass = im.data();
        view.inv_inertia = ii.data();
        view.mesh_id = mesh_id.data();
        view.mesh_scale = scale.data();
        view.albedo = albedo.data();
        view.mesh_vert_off = mesh_vert_off.data();
        view.mesh_verts = verts.data();
        view.mesh_tri_off = mesh_tri_off.data();
        view.mesh_tris = mesh_tris.data();
        view.cam_off = cam_off.data();
        view.cam_w = cam_w.data();
        view.cam_h = cam_h.data();
        view.cam_eye = eye.data();
        view.cam_right = right.data();
        view.cam_up = up.data();
        view.cam_fwd = fwd.data();
        view.cam_fpy = fpy.data();
    }
};

struct Job {
    int64_t id = 0;
    SceneCopy* scene = nullptr;   // until admitted
    vuda_sim_params params{};
    int64_t est_bytes = 0, bytes = 0;
    vuda_env_t env = nullptr;
    vuda_frame frame{};
    void* frame_mem = nullptr;
    int desc = -1;
    std::vector<int32_t> cam_h, cam_w, body_off;
    std::deque<uint64_t> queued;
    int inflight = 0;
    bool removing = false;
};

struct Req {
    int64_t job;
    double t_submit = 0, t_start = 0;
    int64_t step = 0;
};

struct Iter {
    int64_t no = 0;               // iteration number; its events are ring entries no % kRing
    std::vector<uint64_t> reqs;
    double t_launch = 0;
};

// Pinned host + device buffer pair that grows on demand.
template <typename T>
struct Buf {
    T* h = nullptr;
    T* d = nullptr;
    size_t cap = 0;
    cudaError_t reserve(size_t n) {
        if (n <= cap) return cudaSuccess;
        size_t c = std::max(n, cap * 2 + 64);
        if (h) cudaFreeHost(h);
        if (d) cudaFree(d);
        h = nullptr;
        d = nullptr;
        cap = 0;
        cudaError_t e = cudaMallocHost((void**)&h, c * sizeof(T));
        if (e == cudaSuccess) e = cudaMalloc((void**)&d, c * sizeof(T));
        if (e == cudaSuccess) cap = c;
        return e;
    }
    void release() {
        if (h) cudaFreeHost(h);
        if (d) cudaFree(d);
        h = nullptr;
        d = nullptr;
        cap = 0;
    }
};

}  // namespace

struct vuda_server {
    vuda_serve_opts o{};
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    std::string fatal;
    int64_t next_job = 1;
    uint64_t next_req = 1;
    std::map<int64_t, Job*> jobs;
    std::deque<int64_t> admit_queue;
    std::unordered_map<uint64_t, Req> reqs;
    std::deque<vuda_result> results;
    int64_t used_bytes = 0, peak_bytes = 0;
    int64_t iterations = 0, batched = 0, completed = 0;
    int max_batch = 0;
    // device side
    DevBatch* descs = nullptr;
    std::vector<int> free_desc;
    cudaStream_t sim_s = nullptr, ren_s = nullptr;
    // physics size classes after the first run on streams of their own,
    // forked from and joined back into sim_s (they hold different jobs)
    cudaStream_t cls_s[2] = {nullptr, nullptr};
    cudaEvent_t cls_fork = nullptr, cls_join[2] = {nullptr, nullptr};
    int* counters = nullptr;
    int sms = 0;
    std::deque<Iter> inflight;
    static constexpr int kRing = 4;   // > max_inflight: a ring entry is reused only after its iteration finished
    cudaEvent_t ev_sim[kRing] = {}, ev_done[kRing] = {};
    int64_t iter_no = 0;
    Buf<int2> sim_items[kRing];
    Buf<int4> ren_items[kRing];
    Buf<int2> shade_items[kRing];
    Buf<TiledJob> tile_jobs[kRing];   // jobs on the tiled path: their device items and list positions
    // host-side fault injection, read from the environment at creation (no
    // GPU fault is ever made): VUDA_FAULT_REJECT_JOB=<id> refuses that job's
    // admission (its requests fail with VUDA_ERR_INVALID); VUDA_FAULT_OOM_JOB
    // =<id> makes its admission fail as if its device memory could not be
    // allocated (VUDA_ERR_OOM, nothing allocated); VUDA_FAULT_STALL_MS=<ms>
    // with VUDA_FAULT_STALL_EVERY=<n> (default 1) stalls the worker that
    // builds and launches batches for ms before every n-th launch
    int64_t fault_reject_job = -1, fault_oom_job = -1;
    int fault_stall_ms = 0, fault_stall_every = 1;
};

namespace {

void release_job_device(Job* j) {
    if (j->env) vuda_env_destroy(j->env);
    j->env = nullptr;
    if (j->frame_mem) cudaFree(j->frame_mem);
    j->frame_mem = nullptr;
}

// Admit waiting jobs in arrival order while they fit the budget.  Called
// with the lock held.
void admit(vuda_server* s) {
    while (!s->admit_queue.empty() && !s->free_desc.empty()) {
        auto it = s->jobs.find(s->admit_queue.front());
        if (it == s->jobs.end()) {
            s->admit_queue.pop_front();
            continue;
        }
        Job* j = it->second;
        if (s->o.hbm_budget_bytes > 0 && s->used_bytes + j->est_bytes > s->o.hbm_budget_bytes) break;
        s->admit_queue.pop_front();
        vuda_env_opts eo{};
        eo.device = s->o.device;
        eo.render_path = VUDA_RENDER_AUTO;   // tiled where its scratch fits, else the band work list
        vuda_status st;
        if (j->id == s->fault_reject_job)
            st = VUDA_ERR_INVALID;           // injected: admission refused
        else if (j->id == s->fault_oom_job)
            st = VUDA_ERR_OOM;               // injected: the job's allocation failed
        else
            st = vuda_env_create(&j->scene->view, &j->params, &eo, &j->env);
        if (st == VUDA_OK) {
            size_t P = (size_t)j->env->P;
            size_t fb = P * 3 + P * 4 + P * 4 + 256;
            if (cudaMalloc(&j->frame_mem, fb) != cudaSuccess) st = VUDA_ERR_OOM;
        }
        if (st != VUDA_OK) {
            // the job cannot run: fail its queued requests
            for (uint64_t r : j->queued) {
                vuda_result res{};
                res.req_id = r;
                res.job_id = j->id;
                res.status = st;
                res.t_submit_ms = s->reqs[r].t_submit;
                res.t_done_ms = now_ms();
                s->results.push_back(res);
                s->reqs.erase(r);
            }
            j->queued.clear();
            release_job_device(j);
            j->removing = true;
            continue;
        }
        uint8_t* base = (uint8_t*)j->frame_mem;
        size_t P = (size_t)j->env->P;
        j->frame.depth = (float*)base;
        j->frame.triid = (uint32_t*)(base + 4 * P);
        j->frame.rgb = base + 8 * P;
        j->bytes = j->env->bytes + (int64_t)(P * 11);
        j->desc = s->free_desc.back();
        s->free_desc.pop_back();
        DevBatch d = j->env->d;
        d.frame = j->frame;
        cudaMemcpy(s->descs + j->desc, &d, sizeof(DevBatch), cudaMemcpyHostToDevice);
        j->cam_w.assign(j->scene->cam_w.begin(), j->scene->cam_w.end());
        j->body_off.assign(j->scene->body_off.begin(), j->scene->body_off.end());
        j->cam_h.assign(j->scene->cam_h.begin(), j->scene->cam_h.end());
        delete j->scene;
        j->scene = nullptr;
        s->used_bytes += j->bytes;
        s->peak_bytes = std::max(s->peak_bytes, s->used_bytes);
    }
}

void retire_job(vuda_server* s, Job* j) {
    if (j->desc >= 0) s->free_desc.push_back(j->desc);
    s->used_bytes -= j->bytes;
    release_job_device(j);
    delete j->scene;
    s->jobs.erase(j->id);
    delete j;
}

// Launch one iteration with one request of every job in `batch`.
bool launch_iteration(vuda_server* s, const std::vector<std::pair<Job*, uint64_t>>& batch) {
    const int64_t no = s->iter_no;
    const int slot_buf = (int)(no % vuda_server::kRing);
    // jobs on the tiled path (created with the default tile size and bin
    // limit) render through the tiled work lists, the others through the band
    // work list
    auto tiled = [](const Job* j) {
        return j->env->tiled && j->env->tile_size == tiled_default_tile() &&
               j->env->bin_limit == tiled_default_bin_limit();
    };
    int max_bodies = 1, max_mcpb = 1, max_w = 1, max_h = 1;
    int any_feat = 0;   // optional contact tests of any job of the batch: the physics variant with them
    size_t nsim = 0, nshade = 0, ntj = 0;
    for (auto& pr : batch) {
        Job* j = pr.first;
        max_bodies = std::max(max_bodies, j->env->max_bodies);
        max_mcpb = std::max(max_mcpb, j->params.max_contacts_per_body);
        any_feat |= sim_features(j->env->sc);
        nsim += j->env->E;
        if (tiled(j)) {
            ntj++;
            continue;
        }
        for (int w : j->cam_w) max_w = std::max(max_w, w);
        for (int h : j->cam_h) max_h = std::max(max_h, h);
        nshade += j->env->B + j->env->E;
    }
    const int br = render_default_band_rows(max_w, max_h);
    size_t nren = 0;
    for (auto& pr : batch)
        if (!tiled(pr.first))
            for (size_t c = 0; c < pr.first->cam_h.size(); c++) nren += (pr.first->cam_h[c] + br - 1) / br;
    Buf<int2>& si = s->sim_items[slot_buf];
    Buf<int4>& ri = s->ren_items[slot_buf];
    Buf<int2>& hi = s->shade_items[slot_buf];
    Buf<TiledJob>& tj = s->tile_jobs[slot_buf];
    if (si.reserve(nsim) != cudaSuccess || ri.reserve(nren) != cudaSuccess || hi.reserve(nshade) != cudaSuccess ||
        tj.reserve(ntj) != cudaSuccess) {
        s->fatal = "serving item buffers: out of memory";
        return false;
    }
    // items, largest environments and bands first
    std::vector<std::pair<int, int2>> sims;
    sims.reserve(nsim);
    size_t a = 0, b = 0, c2 = 0, kj = 0;
    int ncams = 0, nitems = 0;
    for (auto& pr : batch) {
        Job* j = pr.first;
        const int slot = (int)(j->env->steps & 1);
        const int tag = j->desc | (slot << 24);
        const std::vector<int32_t>& boff = j->body_off;
        for (int e = 0; e < j->env->E; e++) sims.push_back({boff[e + 1] - boff[e], make_int2(tag, e)});
        if (tiled(j)) {
            tj.h[kj++] = TiledJob{j->env->tcams, j->env->titems, j->env->ts, ncams, nitems, tag, 0};
            ncams += j->env->C;
            nitems += j->env->ntitems;
            continue;
        }
        int cam = 0;
        for (size_t cc = 0; cc < j->cam_h.size(); cc++, cam++)
            for (int y = 0; y < j->cam_h[cc]; y += br) ri.h[b++] = make_int4(tag, cam, y, 0);
        for (int u = 0; u < j->env->B + j->env->E; u++) hi.h[c2++] = make_int2(tag, u);
    }
    {
        // largest environments first: a stable counting sort by body count
        // (the same order as a stable comparison sort, in linear time)
        int maxb = 0;
        for (auto& p : sims) maxb = std::max(maxb, p.first);
        std::vector<size_t> start((size_t)maxb + 2, 0);
        for (auto& p : sims) start[(size_t)(maxb - p.first) + 1]++;
        for (size_t k = 1; k < start.size(); k++) start[k] += start[k - 1];
        std::vector<std::pair<int, int2>> sorted(sims.size());
        for (auto& p : sims) sorted[start[(size_t)(maxb - p.first)]++] = p;
        sims.swap(sorted);
    }
    for (auto& p : sims) si.h[a++] = p.second;

    // physics by size class (the items are sorted by body count, so each class
    // is a contiguous range): more than kWideBodies bodies on 512-thread CTAs,
    // then up to kWideBodies and up to 32 on 128-thread CTAs, each with the
    // shared-memory layout of its own largest environment
    struct Cls {
        size_t off = 0, n = 0;
        int nb = 0, smem = 0, grid = 0;
        bool wide = false;
    };
    Cls cls[3];
    {
        const int bounds[3] = {1 << 30, kWideBodies, 32};
        size_t q = 0;
        for (int k = 0; k < 3; k++) {
            const int lo = k == 2 ? 0 : bounds[k + 1];
            cls[k].off = q;
            cls[k].wide = k == 0;
            while (q < sims.size() && sims[q].first > lo) {
                cls[k].nb = std::max(cls[k].nb, sims[q].first);
                q++;
            }
            cls[k].n = q - cls[k].off;
            if (!cls[k].n) continue;
            cls[k].smem = cls[k].wide ? wide::phys_smem_bytes_default(cls[k].nb, max_mcpb)
                                      : phys_smem_bytes_default(cls[k].nb, max_mcpb);
            const int per_sm = cls[k].wide ? wide::sim_ctas_per_sm(cls[k].smem) : sim_ctas_per_sm(cls[k].smem);
            cls[k].grid = std::max(1, std::min((int)cls[k].n, s->sms * per_sm));
        }
    }
    (void)max_bodies;
    const int ren_grid = std::max(1, std::min((int)nren, s->sms * render_ctas_per_sm(br, max_w)));
    Iter it;
    it.no = no;
    it.t_launch = now_ms();
    cudaEvent_t ev_sim = s->ev_sim[slot_buf], ev_done = s->ev_done[slot_buf];
    cudaError_t e = cudaSuccess;
    // pose slots are reused two iterations later: wait for that render
    if (no >= 2) e = cudaStreamWaitEvent(s->sim_s, s->ev_done[(no - 2) % vuda_server::kRing], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(si.d, si.h, nsim * sizeof(int2), cudaMemcpyHostToDevice, s->sim_s);
    // the classes side by side when more than one has work: the small
    // environments fill the SMs around the long chains of the largest
    int nbusy = 0;
    for (int k = 0; k < 3; k++) nbusy += cls[k].n ? 1 : 0;
    const bool fork = nbusy > 1 && s->cls_s[0] && s->cls_s[1];
    if (fork && e == cudaSuccess) {
        e = cudaEventRecord(s->cls_fork, s->sim_s);
        for (int q = 0; q < 2 && e == cudaSuccess; q++) e = cudaStreamWaitEvent(s->cls_s[q], s->cls_fork, 0);
    }
    int lane = 0;   // the stream the next busy class goes to: sim_s, then cls_s[0], cls_s[1]
    bool used[2] = {false, false};
    for (int k = 0; k < 3 && e == cudaSuccess; k++) {
        if (!cls[k].n) continue;
        cudaStream_t cs = s->sim_s;
        if (fork && lane > 0) {
            cs = s->cls_s[lane - 1];
            used[lane - 1] = true;
        }
        lane++;
        const int2* items = si.d + cls[k].off;
        e = cls[k].wide ? wide::launch_sim_items(s->descs, items, (int)cls[k].n, s->counters + 2 + k, cls[k].grid,
                                                 cls[k].smem, cls[k].nb, nullptr, SmGate{nullptr, 0}, any_feat, cs)
                        : launch_sim_items(s->descs, items, (int)cls[k].n, s->counters + 2 + k, cls[k].grid,
                                           cls[k].smem, cls[k].nb, nullptr, SmGate{nullptr, 0}, any_feat, cs);
    }
    for (int q = 0; q < 2 && fork && e == cudaSuccess; q++) {
        if (!used[q]) continue;
        e = cudaEventRecord(s->cls_join[q], s->cls_s[q]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s->sim_s, s->cls_join[q], 0);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev_sim, s->sim_s);
    if (e == cudaSuccess && nren)
        e = cudaMemcpyAsync(ri.d, ri.h, nren * sizeof(int4), cudaMemcpyHostToDevice, s->ren_s);
    if (e == cudaSuccess && nshade)
        e = cudaMemcpyAsync(hi.d, hi.h, nshade * sizeof(int2), cudaMemcpyHostToDevice, s->ren_s);
    if (e == cudaSuccess && ntj)
        e = cudaMemcpyAsync(tj.d, tj.h, ntj * sizeof(TiledJob), cudaMemcpyHostToDevice, s->ren_s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->ren_s, ev_sim, 0);
    if (e == cudaSuccess && (nren || nshade))
        e = launch_render_list(s->descs, ri.d, (int)nren, s->counters + 1, ren_grid, hi.d, (int)nshade, br, max_w,
                               nullptr, SmGate{nullptr, 0}, s->ren_s);
    if (e == cudaSuccess && ntj) e = launch_render_tiled_list(s->descs, tj.d, (int)ntj, ncams, nitems, s->ren_s);
    if (e == cudaSuccess) e = cudaEventRecord(ev_done, s->ren_s);
    if (e != cudaSuccess) {
        s->fatal = std::string("serving launch: ") + cudaGetErrorString(e);
        return false;
    }
    s->iter_no++;
    for (auto& pr : batch) {
        pr.first->env->steps++;
        it.reqs.push_back(pr.second);
    }
    s->inflight.push_back(it);
    return true;
}

void worker_main(vuda_server* s) {
    cudaSetDevice(s->o.device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        // completions, in order
        while (!s->inflight.empty() &&
               cudaEventQuery(s->ev_done[s->inflight.front().no % vuda_server::kRing]) == cudaSuccess) {
            Iter it = s->inflight.front();
            s->inflight.pop_front();
            double t = now_ms();
            for (uint64_t r : it.reqs) {
                auto rq = s->reqs.find(r);
                if (rq == s->reqs.end()) continue;
                vuda_result res{};
                res.req_id = r;
                res.job_id = rq->second.job;
                res.status = VUDA_OK;
                res.t_submit_ms = rq->second.t_submit;
                res.t_start_ms = rq->second.t_start;
                res.t_done_ms = t;
                res.step = rq->second.step;
                s->results.push_back(res);
                auto jb = s->jobs.find(rq->second.job);
                if (jb != s->jobs.end()) jb->second->inflight--;
                s->reqs.erase(rq);
                s->completed++;
            }
            s->cv.notify_all();
        }
        // retire jobs marked for removal once idle
        for (auto it = s->jobs.begin(); it != s->jobs.end();) {
            Job* j = it->second;
            ++it;
            if (j->removing && j->inflight == 0 && j->queued.empty()) retire_job(s, j);
        }
        admit(s);
        // one request of every admitted job that has one, if a slot is free
        std::vector<std::pair<Job*, uint64_t>> batch;
        if ((int)s->inflight.size() < s->o.max_inflight) {
            double t = now_ms();
            for (auto& kv : s->jobs) {
                Job* j = kv.second;
                if (!j->env || j->queued.empty()) continue;
                uint64_t r = j->queued.front();
                j->queued.pop_front();
                j->inflight++;
                Req& rq = s->reqs[r];
                rq.t_start = t;
                rq.step = j->env->steps;
                batch.push_back({j, r});
                if (s->o.max_batch_jobs > 0 && (int)batch.size() >= s->o.max_batch_jobs) break;
            }
        }
        if (!batch.empty()) {
            if (s->fault_stall_ms > 0 && (s->iterations + 1) % s->fault_stall_every == 0) {
                // injected: the producer of launches stalls (the lock is
                // released: clients keep submitting and polling)
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::milliseconds(s->fault_stall_ms));
                lk.lock();
            }
            if (!launch_iteration(s, batch)) break;
            s->iterations++;
            s->batched += (int64_t)batch.size();
            s->max_batch = std::max(s->max_batch, (int)batch.size());
            continue;
        }
        if (s->inflight.empty())
            s->cv.wait_for(lk, std::chrono::milliseconds(2));
        else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
    s->cv.notify_all();
}

}  // namespace

extern "C" {

vuda_status vuda_serve_create(const vuda_serve_opts* opts, vuda_server_t* out) {
    if (!opts || !out) return (set_error("null argument"), VUDA_ERR_INVALID);
    *out = nullptr;
    vuda_serve_opts o = *opts;
    if (o.max_jobs <= 0) o.max_jobs = 64;
    if (o.max_jobs > 4096) return (set_error("max_jobs must be at most 4096"), VUDA_ERR_INVALID);
    if (o.max_inflight <= 0) o.max_inflight = 2;
    if (o.max_inflight > vuda_server::kRing - 1) o.max_inflight = vuda_server::kRing - 1;
    if (o.hbm_budget_bytes < 0) return (set_error("negative HBM budget"), VUDA_ERR_INVALID);
    cudaError_t e = cudaSetDevice(o.device);
    if (e != cudaSuccess) return (set_error(std::string("cudaSetDevice: ") + cudaGetErrorString(e)), VUDA_ERR_CUDA);
    vuda_server* s = new vuda_server();
    s->o = o;
    e = cudaMalloc(&s->descs, sizeof(DevBatch) * o.max_jobs);
    if (e == cudaSuccess) e = cudaMalloc(&s->counters, 5 * sizeof(int));   // render, then one per physics size class
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->sim_s, cudaStreamNonBlocking);
    if (e == cudaSuccess && o.serialized) s->ren_s = s->sim_s;
    else if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->ren_s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, o.device);
    for (int q = 0; q < 2 && e == cudaSuccess; q++) {
        e = cudaStreamCreateWithFlags(&s->cls_s[q], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->cls_join[q], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->cls_fork, cudaEventDisableTiming);
    for (int k = 0; k < vuda_server::kRing && e == cudaSuccess; k++) {
        e = cudaEventCreateWithFlags(&s->ev_sim[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_done[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        set_error(std::string("serving setup: ") + cudaGetErrorString(e));
        if (s->descs) cudaFree(s->descs);
        if (s->counters) cudaFree(s->counters);
        if (s->ren_s && s->ren_s != s->sim_s) cudaStreamDestroy(s->ren_s);
        if (s->sim_s) cudaStreamDestroy(s->sim_s);
        for (int k = 0; k < vuda_server::kRing; k++) {
            if (s->ev_sim[k]) cudaEventDestroy(s->ev_sim[k]);
            if (s->ev_done[k]) cudaEventDestroy(s->ev_done[k]);
        }
        for (int q = 0; q < 2; q++) {
            if (s->cls_s[q]) cudaStreamDestroy(s->cls_s[q]);
            if (s->cls_join[q]) cudaEventDestroy(s->cls_join[q]);
        }
        if (s->cls_fork) cudaEventDestroy(s->cls_fork);
        delete s;
        return VUDA_ERR_CUDA;
    }
    for (int k = o.max_jobs - 1; k >= 0; k--) s->free_desc.push_back(k);
    auto env_int = [](const char* name, long long dflt) {
        const char* v = std::getenv(name);
        return v && *v ? std::atoll(v) : dflt;
    };
    s->fault_reject_job = env_int("VUDA_FAULT_REJECT_JOB", -1);
    s->fault_oom_job = env_int("VUDA_FAULT_OOM_JOB", -1);
    s->fault_stall_ms = (int)std::max(0LL, env_int("VUDA_FAULT_STALL_MS", 0));
    s->fault_stall_every = (int)std::max(1LL, env_int("VUDA_FAULT_STALL_EVERY", 1));
    s->worker = std::thread(worker_main, s);
    *out = s;
    return VUDA_OK;
}

vuda_status vuda_serve_destroy(vuda_server_t s) {
    if (!s) return VUDA_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->o.device);
    cudaDeviceSynchronize();
    for (auto& kv : s->jobs) {
        release_job_device(kv.second);
        delete kv.second->scene;
        delete kv.second;
    }
    for (int k = 0; k < vuda_server::kRing; k++) {
        if (s->ev_sim[k]) cudaEventDestroy(s->ev_sim[k]);
        if (s->ev_done[k]) cudaEventDestroy(s->ev_done[k]);
    }
    for (int k = 0; k < vuda_server::kRing; k++) {
        s->sim_items[k].release();
        s->ren_items[k].release();
        s->shade_items[k].release();
        s->tile_jobs[k].release();
    }
    if (s->ren_s && s->ren_s != s->sim_s) cudaStreamDestroy(s->ren_s);
    if (s->sim_s) cudaStreamDestroy(s->sim_s);
    for (int q = 0; q < 2; q++) {
        if (s->cls_s[q]) cudaStreamDestroy(s->cls_s[q]);
        if (s->cls_join[q]) cudaEventDestroy(s->cls_join[q]);
    }
    if (s->cls_fork) cudaEventDestroy(s->cls_fork);
    cudaFree(s->descs);
    cudaFree(s->counters);
    delete s;
    return VUDA_OK;
}

vuda_status vuda_serve_add_job(vuda_server_t s, const vuda_scene* scene, const vuda_sim_params* params,
                               int64_t* job_id) {
    if (!s || !scene || !params || !job_id) return (set_error("null argument"), VUDA_ERR_INVALID);
    int64_t est = 0;
    vuda_status st = env_estimate_bytes(scene, params, &est);
    if (st != VUDA_OK) return st;
    if (s->o.hbm_budget_bytes > 0 && est > s->o.hbm_budget_bytes) {
        set_error("job needs " + std::to_string(est) + " bytes, more than the whole HBM budget");
        return VUDA_ERR_OOM;
    }
    Job* j = new Job();
    j->scene = new SceneCopy(*scene);
    j->params = *params;
    j->est_bytes = est;
    std::lock_guard<std::mutex> lk(s->mu);
    j->id = s->next_job++;
    s->jobs[j->id] = j;
    s->admit_queue.push_back(j->id);
    *job_id = j->id;
    s->cv.notify_all();
    return VUDA_OK;
}

vuda_status vuda_serve_submit(vuda_server_t s, int64_t job_id, uint64_t* req_id) {
    if (!s || !req_id) return (set_error("null argument"), VUDA_ERR_INVALID);
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->fatal.empty()) return (set_error(s->fatal), VUDA_ERR_CUDA);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end() || it->second->removing) return (set_error("unknown job"), VUDA_ERR_INVALID);
    uint64_t r = s->next_req++;
    Req rq;
    rq.job = job_id;
    rq.t_submit = now_ms();
    s->reqs[r] = rq;
    it->second->queued.push_back(r);
    *req_id = r;
    s->cv.notify_all();
    return VUDA_OK;
}

vuda_status vuda_serve_poll(vuda_server_t s, vuda_result* out, int32_t max, int32_t* n, int32_t wait_ms) {
    if (!s || !n || (max > 0 && !out)) return (set_error("null argument"), VUDA_ERR_INVALID);
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->results.empty() && wait_ms > 0)
        s->cv.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->results.empty() || s->stop; });
    int k = 0;
    while (k < max && !s->results.empty()) {
        out[k++] = s->results.front();
        s->results.pop_front();
    }
    *n = k;
    if (!s->fatal.empty()) return (set_error(s->fatal), VUDA_ERR_CUDA);
    if (k == 0 && wait_ms > 0) return (set_error("no result within wait_ms"), VUDA_ERR_TIMEOUT);
    return VUDA_OK;
}

vuda_status vuda_serve_remove_job(vuda_server_t s, int64_t job_id) {
    if (!s) return (set_error("null argument"), VUDA_ERR_INVALID);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return (set_error("unknown job"), VUDA_ERR_INVALID);
    Job* j = it->second;
    // requests not yet on the GPU are cancelled
    for (uint64_t r : j->queued) {
        vuda_result res{};
        res.req_id = r;
        res.job_id = j->id;
        res.status = VUDA_ERR_BUSY;
        res.t_submit_ms = s->reqs[r].t_submit;
        res.t_done_ms = now_ms();
        s->results.push_back(res);
        s->reqs.erase(r);
    }
    j->queued.clear();
    j->removing = true;
    s->admit_queue.erase(std::remove(s->admit_queue.begin(), s->admit_queue.end(), job_id), s->admit_queue.end());
    s->cv.notify_all();
    return VUDA_OK;
}

vuda_status vuda_serve_job_env(vuda_server_t s, int64_t job_id, vuda_env_t* env, vuda_frame* frame) {
    if (!s || !env) return (set_error("null argument"), VUDA_ERR_INVALID);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return (set_error("unknown job"), VUDA_ERR_INVALID);
    *env = it->second->env;
    if (frame) *frame = it->second->frame;
    return it->second->env ? VUDA_OK : (set_error("job not admitted yet"), VUDA_ERR_BUSY);
}

vuda_status vuda_serve_read_frame(vuda_server_t s, int64_t job_id, uint8_t* rgb, float* depth, uint32_t* triid) {
    if (!s) return (set_error("null argument"), VUDA_ERR_INVALID);
    vuda_frame f{};
    int64_t P = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(job_id);
        if (it == s->jobs.end() || !it->second->env) return (set_error("unknown or waiting job"), VUDA_ERR_INVALID);
        if (it->second->inflight || !it->second->queued.empty()) return (set_error("job busy"), VUDA_ERR_BUSY);
        f = it->second->frame;
        P = it->second->env->P;
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && rgb) e = cudaMemcpy(rgb, f.rgb, 3 * (size_t)P, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && depth) e = cudaMemcpy(depth, f.depth, 4 * (size_t)P, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && triid) e = cudaMemcpy(triid, f.triid, 4 * (size_t)P, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return (set_error(std::string("read frame: ") + cudaGetErrorString(e)), VUDA_ERR_CUDA);
    return VUDA_OK;
}

vuda_status vuda_serve_stats_get(vuda_server_t s, vuda_serve_stats* out) {
    if (!s || !out) return (set_error("null argument"), VUDA_ERR_INVALID);
    std::lock_guard<std::mutex> lk(s->mu);
    out->jobs = (int32_t)s->jobs.size();
    int adm = 0, waiting = 0;
    for (auto& kv : s->jobs) {
        if (kv.second->env) adm++;
        else if (!kv.second->removing) waiting++;
    }
    out->admitted = adm;
    out->waiting = waiting;
    out->iterations = s->iterations;
    out->requests_done = s->completed;
    out->mean_batch = s->iterations ? (double)s->batched / (double)s->iterations : 0.0;
    out->max_batch = s->max_batch;
    out->used_bytes = s->used_bytes;
    out->peak_bytes = s->peak_bytes;
    out->inflight = (int32_t)s->inflight.size();
    return VUDA_OK;
}

}  // extern "C"
