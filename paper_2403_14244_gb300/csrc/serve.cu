// Render server: continuous batching of render requests over resident scenes.
//
// Requests (scene, camera, output image) are queued by igs_serve_submit. A
// scheduler thread admits them in arrival order as soon as a slot (a CUDA
// stream) is free and their frame workspace fits in the caller's HBM pool,
// enqueues igs_project -> igs_bin_sort -> igs_render_fwd on that slot's stream,
// and collects completions with cudaEventQuery. Requests that arrive while
// others run are admitted at once, so their work overlaps on the GPU. The
// entries a request needs are only known after binning: the server sizes the
// capacity from earlier requests of the same scene and image size (15 % margin)
// and, if a request overflows, re-queues it at the head with the capacity it
// reported. A request that can never fit the pool fails with IGS_ERR_CAPACITY.
// With grouping on, the scheduler takes with the head request the other
// requests of its scene among the first kGroupWindow queued (up to max_group
// views) and renders them by one batched chain (igs_render_batch, images then
// copied to each request's output); a group that overflows is split and its
// requests are redone one by one.
// The library allocates no device memory: frames are carved from the pool.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// First-fit sub-allocator over the caller's pool (host-side bookkeeping only).
class Pool {
  public:
    void init(char* base, size_t bytes) {
        base_ = base;
        free_.clear();
        if (bytes) free_[0] = bytes;
        size_ = bytes;
    }
    size_t size() const { return size_; }
    char* take(size_t bytes) {
        bytes = al(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_ += bytes;
                return base_ + off;
            }
        }
        return nullptr;
    }
    void give(char* p, size_t bytes) {
        bytes = al(bytes);
        size_t off = (size_t)(p - base_);
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    size_t used() const { return used_; }

  private:
    char* base_ = nullptr;
    size_t size_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;
};

struct SceneRec {
    igs_scene scene;
    igs_opts opts;
};

constexpr int kMaxGroup = 16;      // views of one grouped chain
constexpr int kGroupWindow = 64;   // queued requests the scheduler looks through for a group
constexpr int kBlendBatch = 64;    // batched blend: one 64-thread CTA per 8 x 8 block (8: persistent)
constexpr int kStatusWords = 4 + kMaxGroup;  // per slot: frame/batch status, then per-view entries

struct Request {
    uint64_t id = 0;
    int32_t scene = 0;
    igs_camera cam{};
    float* img = nullptr;
    int64_t capacity = 0;
    igs_timing t{};
    bool solo = false;  // redo by itself (its group overflowed)
    bool done = false;
};

// Work in flight on one slot: one request, or a group of one scene's requests.
struct Job {
    std::vector<Request*> reqs;
    bool batched = false;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    igs_frame frame{};
    igs_batch batch{};
};

}  // namespace

struct igs_server {
    int device = 0;
    igs_opts opts{};
    Pool pool;
    int max_slots = 1;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<uint32_t*> status_host;  // pinned, kStatusWords per slot
    std::vector<Job*> slot_job;
    std::vector<void*> slot_fanout;  // per slot: the fan-out streams of its batched groups
    int max_group = 1;
    std::vector<SceneRec> scenes;
    std::map<std::tuple<int, int, int>, int64_t> cap_hint;  // (scene, W, H) -> entries
    std::deque<Request*> pending;
    std::map<uint64_t, Request*> all;
    uint64_t next_id = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    std::atomic<int64_t> admitted_bytes_peak{0};
};

namespace {

int64_t frame_bytes(const igs_server* s, const Request* r, int64_t capacity) {
    size_t bytes = 0;
    const SceneRec& sc = s->scenes[r->scene];
    if (igs_frame_layout(sc.scene.n, capacity, &r->cam, &sc.opts, nullptr, &bytes, nullptr) != IGS_OK) return -1;
    return (int64_t)bytes;
}

int64_t capacity_for(igs_server* s, const Request* r) {
    if (r->capacity > 0) return r->capacity;
    auto it = s->cap_hint.find({r->scene, r->cam.width, r->cam.height});
    const int64_t n = s->scenes[r->scene].scene.n;
    int64_t c = it != s->cap_hint.end() ? it->second : std::max<int64_t>(1 << 16, 16 * n);
    return std::min<int64_t>(c, (1 << 30) - 1);
}

// Pool bytes of a group's batch workspace plus its packed images (each view
// with its request's capacity); -1 if it cannot be laid out.
int64_t group_bytes(const igs_server* s, const std::vector<Request*>& g) {
    const SceneRec& sc = s->scenes[g[0]->scene];
    igs_camera cams[kMaxGroup];
    int64_t caps[kMaxGroup];
    int64_t floats = 0;
    for (size_t v = 0; v < g.size(); ++v) {
        cams[v] = g[v]->cam;
        caps[v] = g[v]->capacity;
        floats += 3 * (int64_t)g[v]->cam.width * g[v]->cam.height;
    }
    size_t bytes = 0;
    if (igs_batch_layout(sc.scene.n, (int32_t)g.size(), cams, &sc.opts, caps, kBlendBatch, nullptr, &bytes,
                         nullptr) != IGS_OK)
        return -1;
    return (int64_t)(al(bytes) + al((size_t)floats * 4));
}

void fail_job(igs_server* s, int slot, igs_status e) {
    std::memset(s->status_host[slot], 0, kStatusWords * 4);
    s->status_host[slot][igs::kInfoErr] = (uint32_t)e;
    cudaEventRecord(s->events[slot], s->streams[slot]);
}

// Launch one admitted request on its slot's stream (no host synchronisation).
void launch_single(igs_server* s, Job* j, int slot, const SceneRec& sc) {
    Request* r = j->reqs[0];
    cudaStream_t st = s->streams[slot];
    size_t bytes = j->ws_bytes;
    igs_status e = igs_frame_layout(sc.scene.n, r->capacity, &r->cam, &sc.opts, j->ws, &bytes, &j->frame);
    if (e == IGS_OK) e = igs_project(&sc.scene, &r->cam, &sc.opts, &j->frame, st);
    if (e == IGS_OK) e = igs_bin_sort(&j->frame, &sc.opts, st);
    if (e == IGS_OK) e = igs_render_fwd(&j->frame, &sc.opts, r->img, st);
    if (e == IGS_OK &&
        cudaMemcpyAsync(s->status_host[slot], j->frame.info, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
        e = IGS_ERR_CUDA;
    if (e == IGS_OK && cudaEventRecord(s->events[slot], st) != cudaSuccess) e = IGS_ERR_CUDA;
    if (e != IGS_OK) fail_job(s, slot, e);
}

// Launch one admitted group: one batched chain, then each view's image to its
// request's output, the batch status and the per-view entry totals to the host.
void launch_group(igs_server* s, Job* j, int slot, const SceneRec& sc) {
    cudaStream_t st = s->streams[slot];
    const int V = (int)j->reqs.size();
    igs_camera cams[kMaxGroup];
    int64_t caps[kMaxGroup];
    for (int v = 0; v < V; ++v) {
        cams[v] = j->reqs[v]->cam;
        caps[v] = j->reqs[v]->capacity;
    }
    size_t bytes = 0;
    igs_status e = igs_batch_layout(sc.scene.n, V, cams, &sc.opts, caps, kBlendBatch, j->ws, &bytes, &j->batch);
    float* images = reinterpret_cast<float*>(j->ws + al(bytes));
    j->batch.fanout = s->slot_fanout[slot];  // the slot's fan-out streams, made once
    if (e == IGS_OK) e = igs_batch_set_views(&j->batch, cams, &sc.opts, st);
    s->slot_fanout[slot] = j->batch.fanout;
    if (e == IGS_OK) e = igs_render_batch(&j->batch, &sc.scene, &sc.opts, images, st);
    for (int v = 0; v < V && e == IGS_OK; ++v)
        if (cudaMemcpyAsync(j->reqs[v]->img, images + j->batch.image_offset[v],
                            (size_t)3 * cams[v].width * cams[v].height * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            e = IGS_ERR_CUDA;
    if (e == IGS_OK &&
        (cudaMemcpyAsync(s->status_host[slot], j->batch.info, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st) !=
             cudaSuccess ||
         cudaMemcpyAsync(s->status_host[slot] + 4, j->batch.view_entries, (size_t)V * 4,
                         cudaMemcpyDeviceToHost, st) != cudaSuccess))
        e = IGS_ERR_CUDA;
    if (e == IGS_OK && cudaEventRecord(s->events[slot], st) != cudaSuccess) e = IGS_ERR_CUDA;
    if (e != IGS_OK) fail_job(s, slot, e);
}

void note_entries(igs_server* s, const Request* r, uint32_t entries) {
    auto& h = s->cap_hint[{r->scene, r->cam.width, r->cam.height}];
    h = std::max<int64_t>(h, (int64_t)(entries * 1.15) + 4096);
}

void finish(igs_server* s, Request* r, uint32_t entries, uint32_t err, int group) {
    r->t.done_ns = now_ns();
    r->t.entries = entries;
    r->t.status = (int32_t)err;
    r->t.group = group;
    if (!err) note_entries(s, r, entries);
    r->done = true;
}

// A finished job: results, hints, or the re-queue of what overflowed.
void complete(igs_server* s, int k) {
    Job* j = s->slot_job[k];
    const uint32_t* info = s->status_host[k];
    const uint32_t err = info[igs::kInfoErr];
    s->pool.give(j->ws, j->ws_bytes);
    s->slot_job[k] = nullptr;
    if (j->batched) {
        if (err == IGS_ERR_CAPACITY) {  // split: every request redone by itself, in its queue order
            for (size_t v = j->reqs.size(); v-- > 0;) {
                Request* r = j->reqs[v];
                if ((int64_t)info[4 + v] > r->capacity) note_entries(s, r, info[4 + v]);  // the entries it needs
                r->solo = true;
                r->capacity = 0;  // sized again from the hint
                r->t.retries += 1;
                s->pending.push_front(r);
            }
        } else {
            for (size_t v = 0; v < j->reqs.size(); ++v)
                finish(s, j->reqs[v], err ? 0u : info[4 + v], err, (int)j->reqs.size());
        }
        delete j;
        return;
    }
    Request* r = j->reqs[0];
    delete j;
    if (err == IGS_ERR_CAPACITY && (int64_t)info[igs::kInfoNeed] > r->capacity) {
        // re-queue at the head with the entries the view reported (plus margin),
        // unless that frame could never fit the pool: then this request fails alone
        const int64_t need = std::min<int64_t>((int64_t)(info[igs::kInfoNeed] * 1.15) + 4096, (1 << 30) - 1);
        const int64_t bytes = frame_bytes(s, r, need);
        if (bytes >= 0 && (size_t)bytes <= s->pool.size()) {
            r->capacity = need;
            auto& h = s->cap_hint[{r->scene, r->cam.width, r->cam.height}];
            h = std::max(h, need);
            r->t.retries += 1;
            s->pending.push_front(r);
            return;
        }
    }
    finish(s, r, info[igs::kInfoM], err, 1);
}

// The head request and, with grouping on, the other queued requests of its
// scene among the first kGroupWindow (in queue order, at most max_group).
std::vector<Request*> pick_group(igs_server* s) {
    std::vector<Request*> g{s->pending.front()};
    if (s->max_group < 2 || g[0]->solo) return g;
    int seen = 0;
    for (auto it = std::next(s->pending.begin()); it != s->pending.end() && seen < kGroupWindow &&
                                                   (int)g.size() < s->max_group;
         ++it, ++seen)
        if ((*it)->scene == g[0]->scene && !(*it)->solo) g.push_back(*it);
    return g;
}

void worker_main(igs_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        // completions
        bool progressed = false;
        for (int k = 0; k < s->max_slots; ++k) {
            if (!s->slot_job[k] || cudaEventQuery(s->events[k]) != cudaSuccess) continue;
            complete(s, k);
            progressed = true;
        }
        if (progressed) s->cv_done.notify_all();
        // admissions, in arrival order; a request that does not fit waits (no overtaking,
        // except by the requests a group takes along)
        while (!s->pending.empty()) {
            int slot = -1;
            for (int k = 0; k < s->max_slots; ++k)
                if (!s->slot_job[k]) {
                    slot = k;
                    break;
                }
            if (slot < 0) break;
            std::vector<Request*> g = pick_group(s);
            int64_t gbytes = -1;
            for (Request* q : g) q->capacity = capacity_for(s, q);
            if (g.size() > 1) gbytes = group_bytes(s, g);
            if (gbytes < 0 || (size_t)gbytes > s->pool.size()) g.resize(1);  // alone, if the group cannot fit
            Request* r = g[0];
            const int64_t bytes = g.size() > 1 ? gbytes : frame_bytes(s, r, r->capacity);
            if (bytes < 0 || (size_t)bytes > s->pool.size()) {
                s->pending.pop_front();
                finish(s, r, 0u, IGS_ERR_CAPACITY, 1);
                s->cv_done.notify_all();
                continue;
            }
            char* ws = s->pool.take((size_t)bytes);
            if (!ws) break;  // wait for memory
            for (Request* q : g) s->pending.erase(std::find(s->pending.begin(), s->pending.end(), q));
            Job* j = new Job();
            j->reqs = g;
            j->batched = g.size() > 1;
            j->ws = ws;
            j->ws_bytes = (size_t)bytes;
            s->slot_job[slot] = j;
            const int64_t t_admit = now_ns();
            int64_t used = (int64_t)s->pool.used();
            if (used > s->admitted_bytes_peak) s->admitted_bytes_peak = used;
            const SceneRec sc = s->scenes[r->scene];  // (a copy: add_scene may grow the table meanwhile)
            lk.unlock();
            const int64_t t_start = now_ns();
            for (Request* q : g) {
                q->t.admit_ns = t_admit;
                q->t.start_ns = t_start;
            }
            if (j->batched)
                launch_group(s, j, slot, sc);
            else
                launch_single(s, j, slot, sc);
            lk.lock();
        }
        bool busy = false;
        for (int k = 0; k < s->max_slots; ++k) busy |= s->slot_job[k] != nullptr;
        if (s->stop && !busy && s->pending.empty()) break;
        if (busy)
            s->cv_work.wait_for(lk, std::chrono::microseconds(20));
        else
            s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
}

}  // namespace

extern "C" {

igs_status igs_serve_create(void* pool, size_t pool_bytes, int32_t max_slots, const igs_opts* opts,
                            igs_server** out) {
    if (!out || !opts || max_slots < 1 || max_slots > 64) return IGS_ERR_INVALID_ARG;
    if (!pool && pool_bytes) return IGS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(pool) & 255) return IGS_ERR_INVALID_ARG;
    if (opts->tile != 8 && opts->tile != 16 && opts->tile != 32) return IGS_ERR_INVALID_ARG;
    igs_server* s = new igs_server();
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return IGS_ERR_CUDA;
    }
    s->opts = *opts;
    s->pool.init(static_cast<char*>(pool), pool_bytes);
    s->max_slots = max_slots;
    s->streams.resize(max_slots);
    s->events.resize(max_slots);
    s->status_host.resize(max_slots);
    s->slot_job.assign(max_slots, nullptr);
    s->slot_fanout.assign(max_slots, nullptr);
    for (int k = 0; k < max_slots; ++k) {
        if (cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s->events[k], cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&s->status_host[k], kStatusWords * sizeof(uint32_t)) != cudaSuccess) {
            igs_serve_destroy(s);
            return IGS_ERR_CUDA;
        }
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return IGS_OK;
}

igs_status igs_serve_set_grouping(igs_server* s, int32_t max_views) {
    if (!s || max_views < 1 || max_views > kMaxGroup) return IGS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    s->max_group = max_views;
    return IGS_OK;
}

igs_status igs_serve_add_scene(igs_server* s, const igs_scene* scene, int32_t sh_degree, int32_t param_mode,
                               int32_t* scene_id) {
    if (!s || !scene || !scene_id || sh_degree < -1 || sh_degree > 3 || (param_mode != 0 && param_mode != 1))
        return IGS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    SceneRec rec;
    rec.scene = *scene;
    rec.opts = s->opts;
    rec.opts.sh_degree = sh_degree;
    rec.opts.param_mode = param_mode;
    s->scenes.push_back(rec);
    *scene_id = (int32_t)s->scenes.size() - 1;
    return IGS_OK;
}

igs_status igs_serve_submit(igs_server* s, int32_t scene_id, const igs_camera* cam, float* img_out,
                            uint64_t* req_id) {
    if (!s || !cam || !img_out || !req_id) return IGS_ERR_INVALID_ARG;
    if (cam->width <= 0 || cam->height <= 0 || cam->fx != cam->fy || !(cam->fx > 0.f)) return IGS_ERR_INVALID_ARG;
    Request* r = new Request();
    r->cam = *cam;
    r->img = img_out;
    r->t.arrival_ns = now_ns();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (scene_id < 0 || scene_id >= (int32_t)s->scenes.size()) {
            delete r;
            return IGS_ERR_INVALID_ARG;
        }
        r->scene = scene_id;
        // a request that could never fit the pool is refused at once
        size_t bytes = 0;
        const SceneRec& sc = s->scenes[scene_id];
        if (igs_frame_layout(sc.scene.n, 1, cam, &sc.opts, nullptr, &bytes, nullptr) != IGS_OK) {
            delete r;
            return IGS_ERR_INVALID_ARG;
        }
        if (bytes > s->pool.size()) {
            delete r;
            return IGS_ERR_CAPACITY;
        }
        r->id = s->next_id++;
        s->all[r->id] = r;
        s->pending.push_back(r);
        *req_id = r->id;
    }
    s->cv_work.notify_one();
    return IGS_OK;
}

igs_status igs_serve_poll(igs_server* s, uint64_t req_id, int64_t timeout_ns, igs_timing* t) {
    if (!s) return IGS_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(req_id);
    if (it == s->all.end()) return IGS_ERR_INVALID_ARG;
    Request* r = it->second;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::nanoseconds(std::max<int64_t>(timeout_ns, 0));
    while (!r->done) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !r->done) return IGS_ERR_NOT_READY;
    }
    if (t) *t = r->t;
    const igs_status st = (igs_status)r->t.status;
    s->all.erase(it);
    delete r;
    return st;
}

igs_status igs_serve_stats(igs_server* s, int64_t* pending, int64_t* in_flight, int64_t* pool_used,
                           int64_t* pool_peak) {
    if (!s) return IGS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    int64_t busy = 0;
    for (auto* j : s->slot_job)
        if (j) busy += (int64_t)j->reqs.size();
    if (pending) *pending = (int64_t)s->pending.size();
    if (in_flight) *in_flight = busy;
    if (pool_used) *pool_used = (int64_t)s->pool.used();
    if (pool_peak) *pool_peak = s->admitted_bytes_peak;
    return IGS_OK;
}

void igs_serve_destroy(igs_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (int k = 0; k < (int)s->streams.size(); ++k) {
        if (s->streams[k]) cudaStreamSynchronize(s->streams[k]);
        if (s->streams[k]) cudaStreamDestroy(s->streams[k]);
        if (s->events[k]) cudaEventDestroy(s->events[k]);
        if (s->status_host[k]) cudaFreeHost(s->status_host[k]);
        if (k < (int)s->slot_fanout.size() && s->slot_fanout[k]) {
            igs_batch b;
            std::memset(&b, 0, sizeof b);
            b.fanout = s->slot_fanout[k];
            igs_batch_release(&b);
        }
    }
    for (auto& kv : s->all) delete kv.second;
    delete s;
}

}  // extern "C"
