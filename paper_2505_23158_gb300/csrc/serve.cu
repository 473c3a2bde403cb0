// Request loop: continuous batching of render requests over several slots.
//
// A slot is a worker thread with its own CUDA stream, scratch buffers and
// status words.  Requests are taken in arrival order (optionally released at
// their arrival times); a request is admitted as soon as a slot is free and
// its memory (chunk blocks, scratch growth, image) fits the context's HBM
// budget - if it does not, the request waits until other requests release
// memory (blocks they held, scratch they freed) or its wait limit expires.
// Admitted requests run concurrently: their kernels, the side-stream chunk
// gathers of streamed scenes and the device-to-host image copies overlap on
// the device.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>

#include "internal.cuh"

using namespace lodge;

extern "C" lodge_status lodge_serve(lodge_ctx* ctx, const lodge_request* reqs, int32_t n,
                                    const lodge_serve_opts* opts, lodge_request_result* results) {
    if (!ctx || (n > 0 && (!reqs || !results)) || n < 0 || !opts)
        return fail(LODGE_E_INVALID, "bad argument");
    if (opts->slots < 1 || opts->slots > 64) return fail(LODGE_E_INVALID, "slots must be in 1..64");
    if (opts->batch < 0) return fail(LODGE_E_INVALID, "batch must be >= 0");
    for (int i = 0; i < n; ++i) {
        if (reqs[i].scene < 0 || reqs[i].scene >= (int32_t)ctx->scenes.size() || !ctx->scenes[reqs[i].scene])
            return fail(LODGE_E_INVALID, "request %d names no scene", i);
        if (reqs[i].cam.width <= 0 || reqs[i].cam.height <= 0)
            return fail(LODGE_E_INVALID, "request %d has an empty image", i);
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return fail(LODGE_E_CUDA, "%s", cudaGetErrorString(e));
    // slots 1..S with their own streams (slot 0 stays with the single-call API);
    // in batch mode the step's frames use slots 1..batch on slot 1's stream
    const int need = std::max(opts->slots, std::min(opts->batch, kMaxBlendBatch));
    while ((int)ctx->slots.size() < need + 1) {
        Slot* sl = nullptr;
        lodge_status r = create_slot(ctx, &sl);
        if (r != LODGE_OK) return r;
    }
    for (int w = 1; w <= need; ++w) {   // slots made by lodge_render_batch have no stream yet
        Slot& sl = *ctx->slots[w];
        sl.share_sms = opts->slots > 1;   // requests run side by side
        if (!sl.own) {
            e = cudaStreamCreateWithFlags(&sl.own, cudaStreamNonBlocking);
            if (e != cudaSuccess) return fail(LODGE_E_CUDA, "%s", cudaGetErrorString(e));
        }
    }
    std::vector<size_t> img_off((size_t)n + 1, 0);
    for (int i = 0; i < n; ++i)
        img_off[i + 1] = img_off[i] + (size_t)reqs[i].cam.width * reqs[i].cam.height * 3;
    const double wait_limit = opts->wait_limit_s > 0 ? opts->wait_limit_s : 10.0;
    using clock = std::chrono::steady_clock;
    const auto t0 = clock::now();
    auto now_s = [&] { return std::chrono::duration<double>(clock::now() - t0).count(); };
    std::atomic<int> next{0};
    std::atomic<int> failures{0};

    auto worker = [&](int w) {
        cudaSetDevice(ctx->device);
        Slot& sl = *ctx->slots[w];
        cudaStream_t s = sl.own;
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= n) break;
            const lodge_request& rq = reqs[i];
            lodge_request_result& res = results[i];
            res = lodge_request_result{};
            res.slot = w;
            if (opts->realtime) {
                const double wait = rq.arrival_s - now_s();
                if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(wait));
            }
            res.start_s = now_s();
            Scene* sc = ctx->scenes[rq.scene].get();
            const size_t img_bytes = sizeof(float) * (img_off[i + 1] - img_off[i]);
            const int64_t up0 = sl.uploads;
            lodge_status r;
            for (;;) {
                r = ensure(ctx, sl.ws.img, img_bytes, s);
                if (r == LODGE_OK)
                    r = render_one(ctx, sl, sc, (lodge_mode)rq.mode, rq.cam, sl.ws.img.as<float>(), s,
                                   nullptr, &res.stats, true, nullptr);
                if (r != LODGE_E_BUDGET || now_s() - res.start_s > wait_limit) break;
                // admission by footprint: wait for another request to release memory
                std::unique_lock<std::recursive_mutex> lk(ctx->mu);
                ctx->freed.wait_for(lk, std::chrono::milliseconds(20));
            }
            if (r == LODGE_OK && opts->h_images) {
                e = cudaMemcpyAsync(opts->h_images + img_off[i], sl.ws.img.p, img_bytes,
                                    cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) r = LODGE_E_CUDA;
            }
            res.finish_s = now_s();
            res.status = r;
            res.uploads = (int32_t)(sl.uploads - up0);
            res.step_frames = 1;
            if (r != LODGE_OK) failures.fetch_add(1);
        }
    };
    // steps: the arrived requests (up to opts->batch) composited by one launch
    auto stepper = [&]() {
        cudaSetDevice(ctx->device);
        cudaStream_t s = ctx->slots[1]->own;
        const int B = std::min(opts->batch, kMaxBlendBatch);
        std::vector<int> pending;       // arrived, not yet done (budget retries)
        std::vector<double> first_try((size_t)n, -1.0);
        int next_i = 0;
        while (next_i < n || !pending.empty()) {
            if (pending.empty() && opts->realtime) {
                const double wait = reqs[next_i].arrival_s - now_s();
                if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(wait));
            }
            const double t = now_s();
            while (next_i < n && (!opts->realtime || reqs[next_i].arrival_s <= t)) pending.push_back(next_i++);
            std::vector<int> step(pending.begin(), pending.begin() + std::min<size_t>(pending.size(), (size_t)B));
            std::vector<BatchItem> items(step.size());
            std::vector<int64_t> up0(step.size());
            for (size_t k = 0; k < step.size(); ++k) up0[k] = ctx->slots[1 + k]->uploads;
            lodge_status r = LODGE_OK;
            for (size_t k = 0; k < step.size() && r == LODGE_OK; ++k) {
                const int i = step[k];
                if (first_try[i] < 0) first_try[i] = t;
                Slot& sl = *ctx->slots[1 + k];
                r = ensure(ctx, sl.ws.img, sizeof(float) * (img_off[i + 1] - img_off[i]), s);
                items[k].sc = ctx->scenes[reqs[i].scene].get();
                items[k].mode = (lodge_mode)reqs[i].mode;
                items[k].cam = reqs[i].cam;
                items[k].d_rgb = sl.ws.img.as<float>();
                items[k].st = &results[i].stats;
            }
            if (r == LODGE_OK) r = render_batch(ctx, items.data(), (int)items.size(), 1, s);
            for (size_t k = 0; k < step.size(); ++k) {
                const int i = step[k];
                lodge_request_result& res = results[i];
                lodge_status ri = r != LODGE_OK ? r : items[k].status;
                if (ri == LODGE_E_BUDGET && now_s() - first_try[i] <= wait_limit) continue;  // next step
                if (ri == LODGE_OK && opts->h_images) {
                    e = cudaMemcpyAsync(opts->h_images + img_off[i], ctx->slots[1 + k]->ws.img.p,
                                        sizeof(float) * (img_off[i + 1] - img_off[i]), cudaMemcpyDeviceToHost, s);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                    if (e != cudaSuccess) ri = LODGE_E_CUDA;
                }
                res.start_s = first_try[i];
                res.finish_s = now_s();
                res.status = ri;
                res.slot = (int32_t)k;
                res.uploads = (int32_t)(ctx->slots[1 + k]->uploads - up0[k]);
                res.step_frames = (int32_t)step.size();
                if (ri != LODGE_OK) failures.fetch_add(1);
                pending.erase(std::find(pending.begin(), pending.end(), i));
            }
            if (r == LODGE_E_BUDGET) {   // nothing of the step fitted: wait for memory
                std::unique_lock<std::recursive_mutex> lk(ctx->mu);
                ctx->freed.wait_for(lk, std::chrono::milliseconds(20));
            }
        }
    };
    if (opts->batch > 0) {
        stepper();
    } else {
        std::vector<std::thread> th;
        for (int w = 1; w <= opts->slots; ++w) th.emplace_back(worker, w);
        for (auto& t : th) t.join();
    }
    if (failures.load() > 0)
        return fail(LODGE_E_INVALID, "%d of %d requests failed (see their status)", failures.load(), n);
    return LODGE_OK;
}
