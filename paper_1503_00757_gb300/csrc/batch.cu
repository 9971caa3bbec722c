// Batched registration of many independent image pairs: a native
// host-side executor.  Pairs are independent (one registration each), so the
// GB300 is filled by running several Newton-Krylov solves at once, each on
// its own stream, instead of one solve at a time.
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "internal.h"

struct reg_executor {
    int dev;
    std::vector<std::pair<cudaStream_t, std::map<std::pair<int, int>, reg_ctx*>>> workers;
};

static void executor_free(reg_executor* ex) {
    if (!ex) return;
    for (auto& w : ex->workers) {
        for (auto& kv : w.second) reg_destroy(kv.second);
        if (w.first) cudaStreamDestroy(w.first);
    }
    delete ex;
}

extern "C" int reg_executor_create(int nworkers, reg_executor** out) {
    if (!out) return reg_fail(REG_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nworkers <= 0) nworkers = 8;
    if (nworkers > 256) return reg_fail(REG_ERR_ARG, "nworkers must be <= 256");
    reg_executor* ex = new reg_executor();
    cudaError_t e = cudaGetDevice(&ex->dev);
    if (e != cudaSuccess) {
        delete ex;
        return reg_fail(REG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    }
    ex->workers.resize(nworkers);
    for (auto& w : ex->workers) {
        w.first = nullptr;
        e = cudaStreamCreateWithFlags(&w.first, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            executor_free(ex);
            return reg_fail(REG_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
        }
    }
    *out = ex;
    return REG_OK;
}

extern "C" void reg_executor_destroy(reg_executor* ex) { executor_free(ex); }

extern "C" int reg_executor_solve(reg_executor* ex, reg_batch_item* items, int count, const reg_solve_opts* opts) {
    if (!ex) return reg_fail(REG_ERR_ARG, "executor is NULL");
    if (count < 0 || (count > 0 && !items)) return reg_fail(REG_ERR_ARG, "invalid batch");
    if (count == 0) return REG_OK;
    for (int i = 0; i < count; ++i) {
        if (!items[i].mT || !items[i].mR || !items[i].v) return reg_fail(REG_ERR_ARG, "batch item with a NULL buffer");
        items[i].status = -1;
    }
    const int nworkers = std::min<int>((int)ex->workers.size(), count);
    // FFT tiles of every grid size in the batch (measured once per process and device)
    {
        cudaSetDevice(ex->dev);
        std::map<std::pair<int, int>, int> sizes;  // grid -> largest nt of its pairs
        for (int i = 0; i < count; ++i) {
            int& nt = sizes[std::make_pair(items[i].grid.n1, items[i].grid.n2)];
            nt = std::max(nt, std::min(items[i].nt, 4096));
        }
        for (const auto& kv : sizes) {
            const int st = reg_autotune(reg_grid{kv.first.first, kv.first.second}, std::max(kv.second, 1),
                                        std::min(nworkers, 8), 0, nullptr, nullptr, nullptr, nullptr, nullptr);
            if (st != REG_OK) return st;
        }
    }
    // largest grids first (longest-processing-time-first scheduling)
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (long long)items[a].grid.n1 * items[a].grid.n2 > (long long)items[b].grid.n1 * items[b].grid.n2;
    });
    std::atomic<int> next(0);
    std::mutex err_mu;
    std::string first_err;

    auto run = [&](int w) {
        cudaSetDevice(ex->dev);
        cudaStream_t stream = ex->workers[w].first;
        auto& ctxs = ex->workers[w].second;
        for (;;) {
            const int k = next.fetch_add(1);
            if (k >= count) break;
            reg_batch_item& it = items[order[k]];
            const auto key = std::make_pair(it.grid.n1, it.grid.n2);
            reg_ctx* c = nullptr;
            int st = REG_OK;
            auto f = ctxs.find(key);
            if (f == ctxs.end()) {
                st = reg_create(it.grid, it.nt, it.regnorm, it.beta, it.gamma, it.shear, &c);
                if (st == REG_OK) {
                    reg_set_stream(c, stream);
                    ctxs[key] = c;
                }
            } else {
                c = f->second;
                st = reg_set_params(c, it.nt, it.regnorm, it.beta, it.gamma, it.shear);
            }
            if (st == REG_OK) st = reg_set_images(c, it.mT, it.mR);
            if (st == REG_OK) st = reg_solve(c, it.v, opts, &it.stats);
            if (st == REG_OK && it.want_detgrad) st = reg_detgrad(c, it.v, nullptr, it.detgrad);
            if (st == REG_OK) {
                const cudaError_t se = cudaStreamSynchronize(stream);
                if (se != cudaSuccess) st = reg_fail(REG_ERR_CUDA, cudaGetErrorString(se));
            }
            it.status = st;
            if (st != REG_OK) {
                std::lock_guard<std::mutex> lock(err_mu);
                if (first_err.empty()) first_err = reg_last_error();
            }
        }
    };
    std::vector<std::thread> threads;
    for (int w = 0; w < nworkers; ++w) threads.emplace_back(run, w);
    for (auto& t : threads) t.join();
    for (int k = 0; k < count; ++k) {
        const reg_batch_item& it = items[order[k]];
        if (it.status != REG_OK) {
            const int st = it.status < 0 ? REG_ERR_CUDA : it.status;
            return reg_fail(st, first_err.empty() ? std::string("batch item failed") : first_err);
        }
    }
    return REG_OK;
}

extern "C" int reg_solve_batch(reg_batch_item* items, int count, const reg_solve_opts* opts, int nworkers) {
    if (count < 0 || (count > 0 && !items)) return reg_fail(REG_ERR_ARG, "invalid batch");
    if (count == 0) return REG_OK;
    if (nworkers <= 0) nworkers = 8;
    reg_executor* ex = nullptr;
    int st = reg_executor_create(std::min(nworkers, count), &ex);
    if (st != REG_OK) return st;
    st = reg_executor_solve(ex, items, count, opts);
    executor_free(ex);
    return st;
}
