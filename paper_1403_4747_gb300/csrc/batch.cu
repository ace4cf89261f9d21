// Several meshes behind one operator application.  Each mesh keeps its own
// handle (tree, operators, near field); one call applies the operator of
// Eq. eq_sum (Sec. 3.3 Steps 2-4) to every mesh.  With graphs on, the passes
// of all meshes are one CUDA graph per call, one parallel branch per mesh, so
// meshes too small to fill the GPU overlap instead of running in sequence.
#include "fda_internal.cuh"

#include <new>
#include <string>
#include <vector>

struct fda_batch {
    fda_config cfg;
    cudaStream_t stream = nullptr;  // caller's stream: orders fda_apply_batch
    cudaStream_t cs = nullptr;      // private stream: permutations, graph launch, capture origin
    std::vector<fda_handle *> h;
    std::vector<cudaStream_t> fs;   // one branch stream per mesh
    std::vector<cudaEvent_t> join;  // per mesh: end of its branch
    cudaEvent_t start = nullptr, fork = nullptr, done = nullptr;
    std::string err;
    int state = 0;  // 0 created, 1 trees built, 2 precomputed
    struct graph {
        std::vector<int> key;  // right-hand sides, then per mesh precision | tensor cores << 1
        cudaGraphExec_t exec;  // nullptr: seen once, captured on the next call
        long long kernels;
    };
    std::vector<graph> graphs;
    int graphs_broken = 0;
    long long replays = 0;
};

namespace {

template <typename F>
fda_status bguard(fda_batch *b, F &&f)
{
    try {
        f();
        return FDA_OK;
    } catch (const fda_error &e) {
        b->err = e.msg;
        return e.st;
    } catch (const std::bad_alloc &) {
        b->err = "host allocation failed";
        return FDA_ERR_OOM;
    } catch (...) {
        b->err = "unexpected internal error";
        return FDA_ERR_CUDA;
    }
}

// a mesh's own failure, reported on the batch with the mesh's index
fda_status mesh_status(fda_batch *b, int i, fda_status st)
{
    if (st != FDA_OK) b->err = "mesh " + std::to_string(i) + ": " + fda_last_error(b->h[i]);
    return st;
}

// The per-mesh passes as branches forked from and joined to b->cs: each
// handle runs on its branch stream for the duration of the call.
void branches(fda_batch *b, int nm)
{
    FDA_CUDA(cudaEventRecord(b->fork, b->cs));
    for (size_t i = 0; i < b->h.size(); ++i) {
        fda_handle *h = b->h[i];
        FDA_CUDA(cudaStreamWaitEvent(b->fs[i], b->fork, 0));
        cudaStream_t keep = h->stream;
        h->stream = b->fs[i];
        try {
            fda_apply_sorted(h, h->xs.as<c64d>(), h->ys.as<c64d>(), h->cfg.precision, nm);
        } catch (...) {
            h->stream = keep;
            throw;
        }
        h->stream = keep;
        FDA_CUDA(cudaEventRecord(b->join[i], b->fs[i]));
        FDA_CUDA(cudaStreamWaitEvent(b->cs, b->join[i], 0));
    }
}

// The graph of this call (captured here on the second call with the same
// key), or nullptr when the passes run directly.
fda_batch::graph *batch_graph(fda_batch *b, int nm)
{
    if (!b->cfg.graphs || b->graphs_broken) return nullptr;
    std::vector<int> key{nm};
    for (fda_handle *h : b->h) {
        if (h->timing) return nullptr;  // per-pass timing synchronises inside the passes
        key.push_back(h->cfg.precision | (h->cfg.tensor_cores << 1));
    }
    for (auto &g : b->graphs)
        if (g.key == key) {
            if (g.exec) return &g;
            cudaGraph_t graph = nullptr;
            const long long n0 = fda_launches_so_far();
            bool ok = cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                try {
                    branches(b, nm);
                } catch (...) {
                    ok = false;
                }
                // the captured launches were counted but did not run
                g.kernels = fda_launches_so_far() - n0;
                fda_count_launches(-g.kernels);
                ok = (cudaStreamEndCapture(b->cs, &graph) == cudaSuccess) && ok && graph;
            }
            if (ok) ok = cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess;
            if (graph) cudaGraphDestroy(graph);
            if (!ok) {
                (void)cudaGetLastError();
                g.exec = nullptr;
                b->graphs_broken = 1;
                return nullptr;
            }
            return &g;
        }
    b->graphs.push_back(fda_batch::graph{key, nullptr, 0});  // first call: run directly (builds tile caches)
    return nullptr;
}

}  // namespace

extern "C" {

fda_status fda_create_batch(const fda_config *cfg, int nmesh, fda_batch **out)
{
    if (!out) return FDA_ERR_ARG;
    *out = nullptr;
    if (nmesh < 1 || nmesh > 64) return FDA_ERR_ARG;
    fda_config c;
    if (cfg) c = *cfg; else fda_default_config(&c);
    fda_batch *b = new (std::nothrow) fda_batch();
    if (!b) return FDA_ERR_OOM;
    b->cfg = c;
    b->stream = (cudaStream_t)c.cuda_stream;
    fda_status st = bguard(b, [&] {
        // handles first: an invalid configuration fails here, before any CUDA call
        for (int i = 0; i < nmesh; ++i) {
            fda_handle *h = nullptr;
            fda_status s = fda_create(&c, &h);
            if (s != FDA_OK) throw fda_error{s, "mesh " + std::to_string(i) + ": fda_create failed"};
            b->h.push_back(h);
        }
        FDA_CUDA(cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking));
        FDA_CUDA(cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming));
        FDA_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
        FDA_CUDA(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming));
        for (int i = 0; i < nmesh; ++i) {
            cudaStream_t f = nullptr;
            FDA_CUDA(cudaStreamCreateWithFlags(&f, cudaStreamNonBlocking));
            b->fs.push_back(f);
            cudaEvent_t e = nullptr;
            FDA_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            b->join.push_back(e);
        }
    });
    if (st != FDA_OK) {
        fda_destroy_batch(b);
        return st;
    }
    *out = b;
    return FDA_OK;
}

fda_status fda_build_batch(fda_batch *b, const double *const *verts, const int64_t *nv, const int32_t *const *tris,
                           const int64_t *nt, const double *k)
{
    if (!b) return FDA_ERR_ARG;
    if (b->state != 0) {
        b->err = "fda_build_batch called twice";
        return FDA_ERR_STATE;
    }
    if (!verts || !nv || !tris || !nt || !k) {
        b->err = "invalid fda_build_batch arguments";
        return FDA_ERR_ARG;
    }
    for (size_t i = 0; i < b->h.size(); ++i) {
        fda_status st = fda_build_tree(b->h[i], verts[i], nv[i], tris[i], nt[i], k[i]);
        if (st != FDA_OK) return mesh_status(b, (int)i, st);
    }
    b->state = 1;
    return FDA_OK;
}

fda_status fda_precompute_batch(fda_batch *b)
{
    if (!b) return FDA_ERR_ARG;
    if (b->state != 1) {
        b->err = b->state == 0 ? "fda_precompute_batch before fda_build_batch" : "fda_precompute_batch called twice";
        return FDA_ERR_STATE;
    }
    for (size_t i = 0; i < b->h.size(); ++i) {
        fda_status st = fda_precompute_translations(b->h[i]);
        if (st != FDA_OK) return mesh_status(b, (int)i, st);
    }
    b->state = 2;
    return FDA_OK;
}

fda_status fda_apply_batch(fda_batch *b, const fda_c128 *const *x, fda_c128 *const *y, int nrhs, const int64_t *ld)
{
    if (!b) return FDA_ERR_ARG;
    if (b->state != 2) {
        b->err = "fda_apply_batch before fda_precompute_batch";
        return FDA_ERR_STATE;
    }
    if (!x || !y || !ld || nrhs < 1) {
        b->err = "invalid fda_apply_batch arguments";
        return FDA_ERR_ARG;
    }
    for (size_t i = 0; i < b->h.size(); ++i)
        if (!x[i] || !y[i] || ld[i] < b->h[i]->N) {
            b->err = "invalid fda_apply_batch arguments for mesh " + std::to_string(i);
            return FDA_ERR_ARG;
        }
    return bguard(b, [&] {
        const int mr = std::max(1, b->cfg.max_rhs);
        FDA_CUDA(cudaEventRecord(b->start, b->stream));
        FDA_CUDA(cudaStreamWaitEvent(b->cs, b->start, 0));
        for (int m0 = 0; m0 < nrhs; m0 += mr) {
            const int nm = std::min(mr, nrhs - m0);
            fda_batch::graph *g = batch_graph(b, nm);
            for (size_t i = 0; i < b->h.size(); ++i)
                fda_gather_cols(b->h[i], reinterpret_cast<const c64d *>(x[i]) + (int64_t)m0 * ld[i], ld[i],
                                b->h[i]->xs.as<c64d>(), nm, b->cs);
            if (g) {
                FDA_CUDA(cudaGraphLaunch(g->exec, b->cs));
                ++b->replays;
                fda_count_launches(g->kernels);
            } else {
                branches(b, nm);
            }
            for (size_t i = 0; i < b->h.size(); ++i)
                fda_scatter_cols(b->h[i], b->h[i]->ys.as<c64d>(), reinterpret_cast<c64d *>(y[i]) + (int64_t)m0 * ld[i],
                                 ld[i], nm, b->cs);
        }
        FDA_CUDA(cudaEventRecord(b->done, b->cs));
        FDA_CUDA(cudaStreamWaitEvent(b->stream, b->done, 0));
    });
}

fda_handle *fda_batch_mesh(fda_batch *b, int i)
{
    if (!b || i < 0 || i >= (int)b->h.size()) return nullptr;
    return b->h[i];
}

fda_status fda_get_batch_stats(fda_batch *b, fda_batch_stats *out)
{
    if (!b || !out) return FDA_ERR_ARG;
    *out = fda_batch_stats{};
    out->nmesh = (int)b->h.size();
    out->graph_replays = b->replays;
    out->graph_fallback = b->graphs_broken;
    for (size_t i = 0; i < b->h.size(); ++i) {
        out->n_total += b->h[i]->N;
        if (b->state >= 1) {
            fda_stats s;
            fda_status st = fda_get_stats(b->h[i], &s);
            if (st != FDA_OK) return mesh_status(b, (int)i, st);
            out->device_bytes += (size_t)s.device_bytes;
        }
    }
    return FDA_OK;
}

const char *fda_batch_last_error(const fda_batch *b)
{
    if (!b) return "null batch";
    return b->err.c_str();
}

void fda_destroy_batch(fda_batch *b)
{
    if (!b) return;
    if (b->cs) cudaStreamSynchronize(b->cs);
    for (auto &g : b->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (fda_handle *h : b->h) fda_destroy(h);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    for (cudaStream_t s : b->fs) cudaStreamDestroy(s);
    for (cudaEvent_t e : {b->start, b->fork, b->done})
        if (e) cudaEventDestroy(e);
    if (b->cs) cudaStreamDestroy(b->cs);
    delete b;
}

}  // extern "C"
