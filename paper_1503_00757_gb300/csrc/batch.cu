// Batched registration of many independent image pairs (row a15): a native
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

namespace {
struct Worker {
    cudaStream_t stream = nullptr;
    std::map<std::pair<int, int>, reg_ctx*> ctx;  // per grid size
};
}  // namespace

extern "C" int reg_solve_batch(reg_batch_item* items, int count, const reg_solve_opts* opts, int nworkers) {
    if (count < 0 || (count > 0 && !items)) return reg_fail(REG_ERR_ARG, "invalid batch");
    if (count == 0) return REG_OK;
    if (nworkers <= 0) nworkers = 8;
    if (nworkers > count) nworkers = count;
    for (int i = 0; i < count; ++i) {
        if (!items[i].mT || !items[i].mR || !items[i].v) return reg_fail(REG_ERR_ARG, "batch item with a NULL buffer");
        items[i].status = -1;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return reg_fail(REG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));

    // largest grids first (longest-processing-time-first scheduling)
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (long long)items[a].grid.n1 * items[a].grid.n2 > (long long)items[b].grid.n1 * items[b].grid.n2;
    });
    std::atomic<int> next(0);
    std::vector<Worker> workers(nworkers);
    std::mutex err_mu;
    std::string first_err;

    auto run = [&](int w) {
        cudaSetDevice(dev);
        Worker& W = workers[w];
        if (cudaStreamCreateWithFlags(&W.stream, cudaStreamNonBlocking) != cudaSuccess) return;
        for (;;) {
            const int k = next.fetch_add(1);
            if (k >= count) break;
            reg_batch_item& it = items[order[k]];
            const auto key = std::make_pair(it.grid.n1, it.grid.n2);
            reg_ctx* c = nullptr;
            int st = REG_OK;
            auto f = W.ctx.find(key);
            if (f == W.ctx.end()) {
                st = reg_create(it.grid, it.nt, it.regnorm, it.beta, it.gamma, it.shear, &c);
                if (st == REG_OK) {
                    reg_set_stream(c, W.stream);
                    W.ctx[key] = c;
                }
            } else {
                c = f->second;
                st = reg_set_params(c, it.nt, it.regnorm, it.beta, it.gamma, it.shear);
            }
            if (st == REG_OK) st = reg_set_images(c, it.mT, it.mR);
            if (st == REG_OK) st = reg_solve(c, it.v, opts, &it.stats);
            if (st == REG_OK) {
                const cudaError_t se = cudaStreamSynchronize(W.stream);
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
    for (auto& W : workers) {
        for (auto& kv : W.ctx) reg_destroy(kv.second);
        if (W.stream) cudaStreamDestroy(W.stream);
    }
    for (int k = 0; k < count; ++k) {
        const reg_batch_item& it = items[order[k]];
        if (it.status != REG_OK) {
            const int st = it.status < 0 ? REG_ERR_CUDA : it.status;
            return reg_fail(st, first_err.empty() ? std::string("batch item failed") : first_err);
        }
    }
    return REG_OK;
}
