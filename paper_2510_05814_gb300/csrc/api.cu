// extern "C" entry points of libsmoe.so (declared in include/smoe.h):
// argument checks, workspace layout, and the launch sequences.
#include <cmath>
#include <cstring>
#include <vector>

#include "smoe_internal.cuh"

using namespace smoe;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

int64_t tiles_of(int W, int H, int T) {
    return (int64_t)((W + T - 1) / T) * ((H + T - 1) / T);
}

int64_t scan_blocks_of(int64_t n) { return (n + 4095) / 4096; }

// Workspace regions, in order; `fit` adds the batch table and the lists.
struct Layout {
    size_t rec, rect, tile_cnt, cursor, bsum, long_q, n_long, pair_tmp, acc, huge, n_huge;
    size_t table, tile_off, pair_k, n_pairs, done, work, coef, part;
    size_t kcnt, koff, kbsum, ktot, kn_long, pidx;
    size_t total;
};

Layout layout(int64_t K, int64_t tiles, int64_t pair_cap, int S, int GS, int B, bool fit,
              bool det = false) {
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes); return at; };
    if (fit) L.table = take(sizeof(ImgDev) * (size_t)B);
    L.rec = take(sizeof(float) * (size_t)S * (size_t)K);
    L.rect = take(sizeof(int4) * (size_t)K);
    L.tile_cnt = take(sizeof(int32_t) * (size_t)tiles);
    L.cursor = take(sizeof(int32_t) * (size_t)tiles);
    L.bsum = take(sizeof(long long) * (size_t)scan_blocks_of(tiles));
    L.long_q = take(sizeof(int32_t) * (size_t)tiles);
    L.n_long = take(sizeof(int32_t));
    L.acc = take(sizeof(float) * (size_t)GS * (size_t)K);
    L.huge = take(sizeof(int32_t) * (size_t)K);
    L.n_huge = take(sizeof(int32_t));
    L.pair_tmp = take(sizeof(int32_t) * (size_t)pair_cap);
    if (fit) {
        L.tile_off = take(sizeof(int32_t) * (size_t)(tiles + 1));
        L.pair_k = take(sizeof(int32_t) * (size_t)pair_cap);
        L.n_pairs = take(sizeof(int64_t));
        L.done = take(sizeof(uint32_t));
        L.work = take(sizeof(uint32_t));
        L.coef = take(sizeof(float) * 8 * (size_t)B);
        if (det) {
            L.part = take(sizeof(float) * (size_t)GS * (size_t)pair_cap);
            L.kcnt = take(sizeof(int32_t) * (size_t)K);
            L.koff = take(sizeof(int32_t) * (size_t)(K + 1));
            L.kbsum = take(sizeof(long long) * (size_t)scan_blocks_of(K));
            L.ktot = take(sizeof(int64_t));
            L.kn_long = take(sizeof(int32_t));
            L.pidx = take(sizeof(int32_t) * (size_t)pair_cap);
        }
    }
    L.total = o;
    return L;
}

bool desc_ok(const smoe_desc *d) { return desc_valid(d); }

bool params_ok(const smoe_params *p, const smoe_desc *d) {
    if (!p || p->K < 0 || p->K > 0x7fffffffLL) return false;
    if (p->K == 0) return true;
    if (!p->mu || !p->chol || !p->ea) return false;
    if ((p->eW != nullptr) != (d->expert == 1)) return false;
    return true;
}

Geo make_geo(const smoe_desc *d, int64_t K) {
    Geo g{};
    g.C = d->C;
    g.T = d->tile;
    g.linear = d->expert;
    g.S = rec_stride(d->C, d->expert);
    g.GS = acc_stride(d->C, d->expert);
    g.rbf = d->gate;
    g.qmax = d->qmax;
    g.scale = d->scale;
    g.B = 1;
    g.K_total = K;
    g.tiles_total = tiles_of(d->W, d->H, d->tile);
    g.table = nullptr;
    g.one.W = d->W;
    g.one.H = d->H;
    g.one.tiles_x = (d->W + d->tile - 1) / d->tile;
    g.one.tiles_y = (d->H + d->tile - 1) / d->tile;
    g.one.K = K;
    g.one.k_off = 0;
    g.one.t_off = 0;
    g.one.iters = 1;
    g.one.p.K = K;
    return g;
}

Bufs make_bufs(void *ws, const Layout &L) {
    char *b = static_cast<char *>(ws);
    Bufs w{};
    w.rec = reinterpret_cast<float *>(b + L.rec);
    w.rect = reinterpret_cast<int4 *>(b + L.rect);
    w.tile_cnt = reinterpret_cast<int32_t *>(b + L.tile_cnt);
    w.cursor = reinterpret_cast<int32_t *>(b + L.cursor);
    w.bsum = reinterpret_cast<long long *>(b + L.bsum);
    w.pair_tmp = reinterpret_cast<int32_t *>(b + L.pair_tmp);
    w.long_q = reinterpret_cast<int32_t *>(b + L.long_q);
    w.n_long = reinterpret_cast<int32_t *>(b + L.n_long);
    w.acc = reinterpret_cast<float *>(b + L.acc);
    w.huge = reinterpret_cast<int32_t *>(b + L.huge);
    w.n_huge = reinterpret_cast<int32_t *>(b + L.n_huge);
    return w;
}

bool ws_ok(const void *ws, size_t have, size_t need) {
    return ws && (reinterpret_cast<uintptr_t>(ws) % kAlign) == 0 && have >= need;
}

smoe_status cuda_status(cudaError_t e) { return e == cudaSuccess ? SMOE_OK : SMOE_ERR_CUDA; }

// Fit batch -> Geo (table in ws) + host copy of the table.
bool fit_geo(const smoe_fit_batch *bt, const smoe_fit_image *imgs, Geo *g,
             std::vector<ImgDev> *tab) {
    if (!bt || !imgs || bt->B <= 0) return false;
    if (bt->C != 1 && bt->C != 3) return false;
    if (bt->tile != 8 && bt->tile != 16 && bt->tile != 32) return false;
    if (bt->expert != 0 && bt->expert != 1) return false;
    if (bt->gate != 0 && bt->gate != 1) return false;
    if (!(bt->qmax > 0.0f) || !(bt->qmax <= kMaxQmax) || !bt->step) return false;
    if (bt->loss && bt->hist <= 0) return false;
    int64_t K_total = 0, t_total = 0;
    tab->resize(bt->B);
    for (int b = 0; b < bt->B; ++b) {
        const smoe_fit_image &im = imgs[b];
        if (im.W <= 0 || im.H <= 0 || im.p.K < 0 || !im.target || im.iters < 0) return false;
        const smoe_params *ps[3] = {&im.p, &im.m, &im.v};
        for (const smoe_params *q : ps) {
            if (q->K != im.p.K) return false;
            if (q->K > 0 && (!q->mu || !q->chol || !q->ea)) return false;
            if (q->K > 0 && ((q->eW != nullptr) != (bt->expert == 1))) return false;
            if (q->K > 0 && ((q->logpi != nullptr) != (im.p.logpi != nullptr))) return false;
        }
        ImgDev &d = (*tab)[b];
        d.W = im.W;
        d.H = im.H;
        d.tiles_x = (im.W + bt->tile - 1) / bt->tile;
        d.tiles_y = (im.H + bt->tile - 1) / bt->tile;
        d.K = im.p.K;
        d.k_off = K_total;
        d.t_off = t_total;
        d.target = im.target;
        d.p = im.p;
        d.m = im.m;
        d.v = im.v;
        d.iters = im.iters;
        d.lr_mu0 = im.lr_mu0;
        d.lr_mu1 = im.lr_mu1 > 0.0f ? im.lr_mu1 : im.lr_mu0;
        d.lr_chol = im.lr_chol;
        d.lr_ea = im.lr_ea;
        d.lr_eW = im.lr_eW;
        d.lr_pi = im.lr_pi;
        if (!(d.lr_mu0 > 0.0f)) d.lr_mu0 = d.lr_mu1 = 0.0f;
        d.mu_rho = d.lr_mu0 > 0.0f && d.iters > 1
                       ? std::pow((double)d.lr_mu1 / (double)d.lr_mu0, 1.0 / (double)(d.iters - 1))
                       : 1.0;
        K_total += im.p.K;
        t_total += (int64_t)d.tiles_x * d.tiles_y;
    }
    if (K_total > 0x7fffffffLL || t_total > kMaxTiles) return false;
    // the deterministic mode scans the kernels' pair counts (the prefix sum's capacity)
    if (bt->deterministic && K_total > kMaxTiles) return false;
    Geo &G = *g;
    G = Geo{};
    G.C = bt->C;
    G.T = bt->tile;
    G.linear = bt->expert;
    G.S = rec_stride(bt->C, bt->expert);
    G.GS = acc_stride(bt->C, bt->expert);
    G.rbf = bt->gate;
    G.qmax = bt->qmax;
    G.scale = 1.0f;
    G.B = bt->B;
    G.K_total = K_total;
    G.tiles_total = t_total;
    if (bt->B == 1) {
        G.table = nullptr;
        G.one = (*tab)[0];
    }
    return true;
}

}  // namespace

extern "C" {

int32_t smoe_version(void) { return (1 << 16) | 0; }

smoe_status smoe_workspace_size(const smoe_desc *d, int64_t K, int64_t pair_cap, size_t *bytes) {
    if (!desc_ok(d) || K < 0 || K > 0x7fffffffLL || pair_cap < 0 || pair_cap > 0x7fffffffLL ||
        !bytes)
        return SMOE_ERR_ARG;
    *bytes = layout(K, tiles_of(d->W, d->H, d->tile), pair_cap, rec_stride(d->C, d->expert),
                    acc_stride(d->C, d->expert), 1, false)
                 .total;
    return SMOE_OK;
}

smoe_status smoe_bin(const smoe_desc *d, const smoe_params *p, void *ws, size_t ws_bytes,
                     int32_t *tile_off, int32_t *pair_k, int64_t pair_cap, int64_t *n_pairs,
                     int32_t *status, void *stream) {
    if (!desc_ok(d) || !params_ok(p, d) || !tile_off || !n_pairs || !status)
        return SMOE_ERR_ARG;
    if (pair_cap < 0 || pair_cap > 0x7fffffffLL || (pair_cap > 0 && !pair_k)) return SMOE_ERR_ARG;
    Geo g = make_geo(d, p->K);
    const Layout L = layout(p->K, g.tiles_total, pair_cap, g.S, g.GS, 1, false);
    if (!ws_ok(ws, ws_bytes, L.total)) return SMOE_ERR_WORKSPACE;
    g.one.p = *p;
    Bufs w = make_bufs(ws, L);
    w.tile_off = tile_off;
    w.pair_k = pair_k;
    w.n_pairs = n_pairs;
    w.pair_cap = pair_cap;
    w.status = status;
    return cuda_status(launch_bin(g, w, static_cast<cudaStream_t>(stream)));
}

smoe_status smoe_render(const smoe_desc *d, int64_t K, const void *ws, size_t ws_bytes,
                        const int32_t *tile_off, const int32_t *pair_k, float *y, float *inv_d,
                        const int32_t *status, void *stream) {
    if (!desc_ok(d) || K < 0 || K > 0x7fffffffLL || !tile_off || !y) return SMOE_ERR_ARG;
    Geo g = make_geo(d, K);
    const Layout L = layout(K, g.tiles_total, 0, g.S, g.GS, 1, false);
    // Only the prepared records are read from ws; the lists are the caller's.
    if (!ws_ok(ws, ws_bytes, L.total)) return SMOE_ERR_WORKSPACE;
    Bufs w = make_bufs(const_cast<void *>(ws), L);
    w.tile_off = const_cast<int32_t *>(tile_off);
    w.pair_k = const_cast<int32_t *>(pair_k);
    w.status = const_cast<int32_t *>(status);
    return cuda_status(launch_render(g, w, y, inv_d, static_cast<cudaStream_t>(stream)));
}

smoe_status smoe_render_backward(const smoe_desc *d, const smoe_params *p, void *ws,
                                 size_t ws_bytes, const int32_t *tile_off, const int32_t *pair_k,
                                 const float *y, const float *inv_d, const float *gy,
                                 const float *target, const smoe_params *grad,
                                 const int32_t *status, void *stream) {
    if (!desc_ok(d) || !params_ok(p, d) || !params_ok(grad, d) || grad->K != p->K || !tile_off ||
        !y || !inv_d || (!gy && !target))
        return SMOE_ERR_ARG;
    Geo g = make_geo(d, p->K);
    // Every region this call uses precedes the pair buffer, so the layout of
    // pair_cap = 0 gives the offsets whatever pair_cap the workspace was made for.
    const Layout L = layout(p->K, g.tiles_total, 0, g.S, g.GS, 1, false);
    if (!ws_ok(ws, ws_bytes, L.total)) return SMOE_ERR_WORKSPACE;
    g.one.p = *p;
    Bufs w = make_bufs(ws, L);
    w.tile_off = const_cast<int32_t *>(tile_off);
    w.pair_k = const_cast<int32_t *>(pair_k);
    w.status = const_cast<int32_t *>(status);
    return cuda_status(launch_render_bwd(g, w, y, inv_d, gy, target, *grad,
                                         static_cast<cudaStream_t>(stream)));
}

smoe_status smoe_adam_step(const smoe_params *p, const smoe_params *g, const smoe_params *m,
                           const smoe_params *v, int32_t C, const float lr[4], double b1,
                           double b2, double eps, int32_t step, void *stream) {
    if (!p || !g || !m || !v || !lr || step < 1 || (C != 1 && C != 3)) return SMOE_ERR_ARG;
    const smoe_params *all[4] = {p, g, m, v};
    const bool has_w = p->eW != nullptr, has_pi = p->logpi != nullptr;
    for (const smoe_params *x : all) {
        if (x->K != p->K || x->K < 0) return SMOE_ERR_ARG;
        if (x->K > 0 && (!x->mu || !x->chol || !x->ea)) return SMOE_ERR_ARG;
        if ((x->eW != nullptr) != has_w) return SMOE_ERR_ARG;
        if ((x->logpi != nullptr) != has_pi) return SMOE_ERR_ARG;
    }
    return cuda_status(launch_adam_soa(*p, *g, *m, *v, C, lr, b1, b2, eps, step,
                                       static_cast<cudaStream_t>(stream)));
}

smoe_status smoe_sq_error(const float *y, const float *target, int64_t n, int32_t clamp,
                          double *out, void *stream) {
    if (n < 0 || (n > 0 && (!y || !target)) || !out) return SMOE_ERR_ARG;
    return cuda_status(launch_sq_error(y, target, n, clamp, out, static_cast<cudaStream_t>(stream)));
}

smoe_status smoe_fit_workspace_size(const smoe_fit_batch *batch, const smoe_fit_image *imgs,
                                    int64_t pair_cap, size_t *bytes) {
    Geo g;
    std::vector<ImgDev> tab;
    if (!fit_geo(batch, imgs, &g, &tab) || pair_cap < 0 || pair_cap > 0x7fffffffLL || !bytes)
        return SMOE_ERR_ARG;
    *bytes = layout(g.K_total, g.tiles_total, pair_cap, g.S, g.GS, g.B, true,
                    batch->deterministic != 0).total;
    return SMOE_OK;
}

static smoe_status fit_bufs(const smoe_fit_batch *batch, const smoe_fit_image *imgs,
                            int64_t pair_cap, void *ws, size_t ws_bytes, int32_t *status,
                            Geo *g, Bufs *w, Layout *L, std::vector<ImgDev> *tab) {
    if (!fit_geo(batch, imgs, g, tab) || pair_cap < 0 || pair_cap > 0x7fffffffLL || !status)
        return SMOE_ERR_ARG;
    *L = layout(g->K_total, g->tiles_total, pair_cap, g->S, g->GS, g->B, true,
                batch->deterministic != 0);
    if (!ws_ok(ws, ws_bytes, L->total)) return SMOE_ERR_WORKSPACE;
    char *b = static_cast<char *>(ws);
    if (g->B > 1) g->table = reinterpret_cast<const ImgDev *>(b + L->table);
    *w = make_bufs(ws, *L);
    w->tile_off = reinterpret_cast<int32_t *>(b + L->tile_off);
    w->pair_k = reinterpret_cast<int32_t *>(b + L->pair_k);
    w->n_pairs = reinterpret_cast<int64_t *>(b + L->n_pairs);
    w->work = reinterpret_cast<uint32_t *>(b + L->work);
    if (batch->deterministic) {
        w->part = reinterpret_cast<float *>(b + L->part);
        w->kcnt = reinterpret_cast<int32_t *>(b + L->kcnt);
        w->koff = reinterpret_cast<int32_t *>(b + L->koff);
        w->kbsum = reinterpret_cast<long long *>(b + L->kbsum);
        w->ktot = reinterpret_cast<int64_t *>(b + L->ktot);
        w->kn_long = reinterpret_cast<int32_t *>(b + L->kn_long);
        w->pidx = reinterpret_cast<int32_t *>(b + L->pidx);
    }
    w->pair_cap = pair_cap;
    w->status = status;
    return SMOE_OK;
}

smoe_status smoe_fit_init(const smoe_fit_batch *batch, const smoe_fit_image *imgs,
                          int64_t pair_cap, void *ws, size_t ws_bytes, int32_t reset,
                          int32_t *status, void *stream) {
    Geo g;
    Bufs w;
    Layout L;
    std::vector<ImgDev> tab;
    smoe_status s = fit_bufs(batch, imgs, pair_cap, ws, ws_bytes, status, &g, &w, &L, &tab);
    if (s != SMOE_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *b = static_cast<char *>(ws);
    cudaError_t e = cudaMemcpyAsync(b + L.table, tab.data(), sizeof(ImgDev) * tab.size(),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.acc, 0, sizeof(float) * g.GS * g.K_total, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b + L.done, 0, sizeof(uint32_t), st);
    if (reset && e == cudaSuccess) {
        for (int bi = 0; bi < batch->B && e == cudaSuccess; ++bi) {
            const smoe_params *mv[2] = {&imgs[bi].m, &imgs[bi].v};
            const int64_t K = imgs[bi].p.K;
            for (const smoe_params *x : mv) {
                if (K == 0) break;
                if (e == cudaSuccess) e = cudaMemsetAsync(x->mu, 0, sizeof(float) * 2 * K, st);
                if (e == cudaSuccess) e = cudaMemsetAsync(x->chol, 0, sizeof(float) * 3 * K, st);
                if (e == cudaSuccess) e = cudaMemsetAsync(x->ea, 0, sizeof(float) * g.C * K, st);
                if (e == cudaSuccess && x->eW)
                    e = cudaMemsetAsync(x->eW, 0, sizeof(float) * 2 * g.C * K, st);
                if (e == cudaSuccess && x->logpi)
                    e = cudaMemsetAsync(x->logpi, 0, sizeof(float) * K, st);
            }
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(batch->step, 0, sizeof(int32_t) * g.B, st);
        if (e == cudaSuccess && batch->loss)
            e = cudaMemsetAsync(batch->loss, 0, sizeof(double) * g.B * batch->hist, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    }
    if (e == cudaSuccess) {
        if (g.B > 1) g.table = reinterpret_cast<const ImgDev *>(b + L.table);
        e = launch_adam_coefs(g, batch->step, batch->b1, batch->b2,
                              reinterpret_cast<float *>(b + L.coef), st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the host table is freed on return
    return cuda_status(e);
}

static cudaError_t fit_phase(const smoe_fit_batch *batch, const Geo &g, const Bufs &w,
                             uint32_t *done, float *coef, int phase, cudaStream_t st) {
    switch (phase) {
        case 0: return launch_bin(g, w, st);
        case 1:
            return launch_fit_tiles(g, w, batch->loss, batch->hist, batch->step,
                                    batch->persistent != 0, st);
        case 2:
            return launch_fit_adam(g, w, batch->b1, batch->b2, batch->eps, batch->step, done,
                                   coef, st);
        default: return cudaErrorInvalidValue;
    }
}

smoe_status smoe_fit(const smoe_fit_batch *batch, const smoe_fit_image *imgs, int64_t pair_cap,
                     void *ws, size_t ws_bytes, int32_t n_iters, int32_t *status, void *stream) {
    Geo g;
    Bufs w;
    Layout L;
    std::vector<ImgDev> tab;
    if (n_iters < 0) return SMOE_ERR_ARG;
    smoe_status s = fit_bufs(batch, imgs, pair_cap, ws, ws_bytes, status, &g, &w, &L, &tab);
    if (s != SMOE_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t *done = reinterpret_cast<uint32_t *>(static_cast<char *>(ws) + L.done);
    float *coef = reinterpret_cast<float *>(static_cast<char *>(ws) + L.coef);
    for (int32_t it = 0; it < n_iters; ++it)
        for (int phase = 0; phase < 3; ++phase)
            if (fit_phase(batch, g, w, done, coef, phase, st) != cudaSuccess) return SMOE_ERR_CUDA;
    return SMOE_OK;
}

smoe_status smoe_fit_phase(const smoe_fit_batch *batch, const smoe_fit_image *imgs,
                           int64_t pair_cap, void *ws, size_t ws_bytes, int32_t phase,
                           int32_t *status, void *stream) {
    Geo g;
    Bufs w;
    Layout L;
    std::vector<ImgDev> tab;
    if (phase < 0 || phase > 2) return SMOE_ERR_ARG;
    smoe_status s = fit_bufs(batch, imgs, pair_cap, ws, ws_bytes, status, &g, &w, &L, &tab);
    if (s != SMOE_OK) return s;
    uint32_t *done = reinterpret_cast<uint32_t *>(static_cast<char *>(ws) + L.done);
    float *coef = reinterpret_cast<float *>(static_cast<char *>(ws) + L.coef);
    return cuda_status(
        fit_phase(batch, g, w, done, coef, phase, static_cast<cudaStream_t>(stream)));
}

smoe_status smoe_fit_gradients(const smoe_fit_batch *batch, const smoe_fit_image *imgs,
                               int64_t pair_cap, void *ws, size_t ws_bytes,
                               const smoe_params *grad, int32_t *status, void *stream) {
    Geo g;
    Bufs w;
    Layout L;
    std::vector<ImgDev> tab;
    smoe_status s = fit_bufs(batch, imgs, pair_cap, ws, ws_bytes, status, &g, &w, &L, &tab);
    if (s != SMOE_OK) return s;
    if (!grad || grad->K != g.K_total) return SMOE_ERR_ARG;
    if (g.K_total > 0 && (!grad->mu || !grad->chol || !grad->ea ||
                          (grad->eW != nullptr) != (batch->expert == 1)))
        return SMOE_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_bin(g, w, st);
    if (e == cudaSuccess)
        e = launch_fit_tiles(g, w, nullptr, 0, batch->step, batch->persistent != 0, st);
    if (e == cudaSuccess) e = launch_fit_grads(g, w, batch->step, *grad, st);
    return cuda_status(e);
}

smoe_status smoe_fit_render_mean(const smoe_fit_batch *batch, const smoe_fit_image *imgs,
                                 int64_t pair_cap, void *ws, size_t ws_bytes, float *y,
                                 int32_t *status, void *stream) {
    Geo g;
    Bufs w;
    Layout L;
    std::vector<ImgDev> tab;
    if (!y) return SMOE_ERR_ARG;
    smoe_status s = fit_bufs(batch, imgs, pair_cap, ws, ws_bytes, status, &g, &w, &L, &tab);
    if (s != SMOE_OK) return s;
    for (int b = 1; b < batch->B; ++b)
        if (imgs[b].W != imgs[0].W || imgs[b].H != imgs[0].H) return SMOE_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_bin(g, w, st);
    if (e == cudaSuccess) e = launch_render_mean(g, w, y, st);
    return cuda_status(e);
}

smoe_status smoe_fit_reorder(const smoe_fit_batch *batch, const smoe_fit_image *imgs,
                             int64_t pair_cap, void *ws, size_t ws_bytes, int32_t *order,
                             int32_t *status, void *stream) {
    Geo g;
    Bufs w;
    Layout L;
    std::vector<ImgDev> tab;
    smoe_status s = fit_bufs(batch, imgs, pair_cap, ws, ws_bytes, status, &g, &w, &L, &tab);
    if (s != SMOE_OK) return s;
    return cuda_status(launch_reorder(g, w, order, static_cast<cudaStream_t>(stream)));
}

smoe_status smoe_scatter_params(const smoe_params *src, const int32_t *index, int64_t base,
                                int32_t C, const smoe_params *dst, void *stream) {
    if (!src || !dst || (C != 1 && C != 3) || src->K < 0 || src->K > 0x7fffffffLL || base < 0)
        return SMOE_ERR_ARG;
    if (src->K > 0 && (!index || !src->mu || !src->chol || !src->ea || !dst->mu || !dst->chol ||
                       !dst->ea))
        return SMOE_ERR_ARG;
    return cuda_status(launch_scatter_params(*src, index, base, src->K, C, *dst,
                                             static_cast<cudaStream_t>(stream)));
}

smoe_status smoe_sharpen(const float *chol_in, float *chol_out, int64_t K, float factor,
                         float qmax, float *qmax_out, void *stream) {
    if (K < 0 || K > 0x7fffffffLL || !(factor > 0.0f) || !std::isfinite(factor) ||
        (K > 0 && (!chol_in || !chol_out)) || !qmax_out)
        return SMOE_ERR_ARG;
    // q_max' = q_max f^2, two FP32 products (f^2 first), so that every point
    // the fitted model includes stays included.
    const float q2 = qmax * (factor * factor);
    if (!(qmax > 0.0f) || !(q2 <= kMaxQmax)) return SMOE_ERR_ARG;
    *qmax_out = q2;
    return cuda_status(launch_scale(chol_in, chol_out, 3 * K, factor,
                                    static_cast<cudaStream_t>(stream)));
}

// Points scratch: cnt, cursor, off (tiles + 1), bsum, n_in, n_long, pt_tile, order.
struct PointLayout {
    size_t cnt, cursor, off, bsum, n_in, n_long, pt_tile, order, total;
};

static PointLayout point_layout(int64_t tiles, int64_t n) {
    PointLayout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes); return at; };
    L.cnt = take(sizeof(int32_t) * (size_t)tiles);
    L.cursor = take(sizeof(int32_t) * (size_t)tiles);
    L.off = take(sizeof(int32_t) * (size_t)(tiles + 1));
    L.bsum = take(sizeof(long long) * (size_t)scan_blocks_of(tiles));
    L.n_in = take(sizeof(int64_t));
    L.n_long = take(sizeof(int32_t));
    L.pt_tile = take(sizeof(int32_t) * (size_t)n);
    L.order = take(sizeof(int32_t) * (size_t)n);
    L.total = o;
    return L;
}

smoe_status smoe_points_workspace_size(const smoe_desc *d, int64_t n_points, size_t *bytes) {
    if (!desc_ok(d) || n_points < 0 || n_points > 0x7fffffffLL || !bytes) return SMOE_ERR_ARG;
    *bytes = point_layout(tiles_of(d->W, d->H, d->tile), n_points).total;
    return SMOE_OK;
}

smoe_status smoe_render_points(const smoe_desc *d, int64_t K, const void *ws, size_t ws_bytes,
                               const int32_t *tile_off, const int32_t *pair_k, int64_t n_points,
                               const float *xy, void *pws, size_t pws_bytes, float *y,
                               float *inv_d, const int32_t *status, void *stream) {
    if (!desc_ok(d) || K < 0 || K > 0x7fffffffLL || !tile_off || n_points < 0 ||
        n_points > 0x7fffffffLL)
        return SMOE_ERR_ARG;
    if (n_points > 0 && (!xy || !y || (reinterpret_cast<uintptr_t>(xy) & 7) != 0))
        return SMOE_ERR_ARG;
    Geo g = make_geo(d, K);
    const Layout L = layout(K, g.tiles_total, 0, g.S, g.GS, 1, false);
    if (!ws_ok(ws, ws_bytes, L.total)) return SMOE_ERR_WORKSPACE;
    const PointLayout PL = point_layout(g.tiles_total, n_points);
    if (!ws_ok(pws, pws_bytes, PL.total)) return SMOE_ERR_WORKSPACE;
    char *b = static_cast<char *>(pws);
    PointBufs pb{};
    pb.cnt = reinterpret_cast<int32_t *>(b + PL.cnt);
    pb.cursor = reinterpret_cast<int32_t *>(b + PL.cursor);
    pb.off = reinterpret_cast<int32_t *>(b + PL.off);
    pb.bsum = reinterpret_cast<long long *>(b + PL.bsum);
    pb.n_in = reinterpret_cast<int64_t *>(b + PL.n_in);
    pb.n_long = reinterpret_cast<int32_t *>(b + PL.n_long);
    pb.pt_tile = reinterpret_cast<int32_t *>(b + PL.pt_tile);
    pb.order = reinterpret_cast<int32_t *>(b + PL.order);
    const float *rec = reinterpret_cast<const float *>(static_cast<const char *>(ws) + L.rec);
    return cuda_status(launch_render_points(g, rec, tile_off, pair_k, n_points, xy, pb, y, inv_d,
                                            status, static_cast<cudaStream_t>(stream)));
}

smoe_status smoe_count_inrange(const smoe_desc *d, int64_t K, const void *ws, size_t ws_bytes,
                               const int32_t *tile_off, const int32_t *pair_k, uint64_t *out,
                               const int32_t *status, void *stream) {
    if (!desc_ok(d) || K < 0 || K > 0x7fffffffLL || !tile_off || !out) return SMOE_ERR_ARG;
    Geo g = make_geo(d, K);
    const Layout L = layout(K, g.tiles_total, 0, g.S, g.GS, 1, false);
    if (!ws_ok(ws, ws_bytes, L.total)) return SMOE_ERR_WORKSPACE;
    const float *rec = reinterpret_cast<const float *>(static_cast<const char *>(ws) + L.rec);
    return cuda_status(launch_count_inrange(g, rec, tile_off, pair_k,
                                            reinterpret_cast<unsigned long long *>(out), status,
                                            static_cast<cudaStream_t>(stream)));
}

// H models rendered on one raster (d, including its scale), as a batch of H
// images of that size: the binning and the averaging launch of Eq. 11.
static bool mean_geo(const smoe_desc *d, const smoe_params *models, int32_t H, Geo *g,
                     std::vector<ImgDev> *tab) {
    if (!desc_ok(d) || !models || H <= 0) return false;
    int64_t K_total = 0;
    const int tx = (d->W + d->tile - 1) / d->tile, ty = (d->H + d->tile - 1) / d->tile;
    tab->assign(H, ImgDev{});
    for (int h = 0; h < H; ++h) {
        if (!params_ok(&models[h], d)) return false;
        if ((models[h].logpi != nullptr) != (models[0].logpi != nullptr)) return false;
        ImgDev &im = (*tab)[h];
        im.W = d->W;
        im.H = d->H;
        im.tiles_x = tx;
        im.tiles_y = ty;
        im.K = models[h].K;
        im.k_off = K_total;
        im.t_off = (int64_t)h * tx * ty;
        im.p = models[h];
        im.iters = 1;
        K_total += models[h].K;
    }
    if (K_total > 0x7fffffffLL || (int64_t)H * tx * ty > kMaxTiles) return false;
    *g = make_geo(d, K_total);
    g->B = H;
    g->tiles_total = (int64_t)H * tx * ty;
    g->table = nullptr;
    if (H == 1) g->one = (*tab)[0];
    return true;
}

smoe_status smoe_render_mean_workspace_size(const smoe_desc *d, const smoe_params *models,
                                            int32_t H, int64_t pair_cap, size_t *bytes) {
    Geo g;
    std::vector<ImgDev> tab;
    if (!mean_geo(d, models, H, &g, &tab) || pair_cap < 0 || pair_cap > 0x7fffffffLL || !bytes)
        return SMOE_ERR_ARG;
    *bytes = layout(g.K_total, g.tiles_total, pair_cap, g.S, g.GS, g.B, true).total;
    return SMOE_OK;
}

smoe_status smoe_render_mean(const smoe_desc *d, const smoe_params *models, int32_t H, void *ws,
                             size_t ws_bytes, int64_t pair_cap, float *y, int32_t *status,
                             void *stream) {
    Geo g;
    std::vector<ImgDev> tab;
    if (!mean_geo(d, models, H, &g, &tab) || pair_cap < 0 || pair_cap > 0x7fffffffLL || !y ||
        !status)
        return SMOE_ERR_ARG;
    const Layout L = layout(g.K_total, g.tiles_total, pair_cap, g.S, g.GS, g.B, true);
    if (!ws_ok(ws, ws_bytes, L.total)) return SMOE_ERR_WORKSPACE;
    char *b = static_cast<char *>(ws);
    Bufs w = make_bufs(ws, L);
    w.tile_off = reinterpret_cast<int32_t *>(b + L.tile_off);
    w.pair_k = reinterpret_cast<int32_t *>(b + L.pair_k);
    w.n_pairs = reinterpret_cast<int64_t *>(b + L.n_pairs);
    w.pair_cap = pair_cap;
    w.status = status;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (H > 1) {
        g.table = reinterpret_cast<const ImgDev *>(b + L.table);
        e = cudaMemcpyAsync(b + L.table, tab.data(), sizeof(ImgDev) * tab.size(),
                            cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the host table is freed on return
    }
    if (e == cudaSuccess) e = launch_bin(g, w, st);
    if (e == cudaSuccess) e = launch_render_mean(g, w, y, st);
    return cuda_status(e);
}

smoe_status smoe_get_status(const int32_t *status, void *stream) {
    if (!status) return SMOE_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return SMOE_ERR_CUDA;
    return (smoe_status)h;
}

}  // extern "C"
