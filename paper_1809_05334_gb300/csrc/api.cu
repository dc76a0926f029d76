// C ABI of the periodic SWG VIE solver (declared in include/vie.h).
//
// vie_solve runs, on the caller's stream:
//   fill   Eq. (2) with the Ewald-summed periodic Green's function (Sec. 2.2)
//   factor the inverse of every domain block A_dd of Eq. (5)-(6)
//   solve  GMRES on diag(A_dd^-1) Z x = diag(A_dd^-1) b, restarted; every restart
//          recomputes the FP64 residual b - Z x (iterative refinement)
//   post   absorbed fraction per domain (Eq. (7)), reflectance, transmittance
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <new>
#include <tuple>
#include <type_traits>
#include <string>
#include <vector>

#include "../../include/vie.h"
#include "blocks.h"
#include "device_math.cuh"
#include "fill.h"
#include "linalg.h"
#include "post.h"
#include "vie_internal.h"

using cplx = std::complex<double>;

namespace vie {
thread_local int64_t g_launches = 0;
}

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    ~DevBuf() { if (p) cudaFree(p); }
    cudaError_t ensure(size_t n) {
        if (n <= bytes && p) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&p, n ? n : 1);
        if (e == cudaSuccess) bytes = n;
        return e;
    }
    template <typename T> T *as() const { return static_cast<T *>(p); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
};

thread_local int64_t *g_h2d_counter = nullptr;   // bytes counter of the solve in progress (host thread local use)

template <typename T>
cudaError_t upload(DevBuf &b, const std::vector<T> &v, cudaStream_t st) {
    if (g_h2d_counter) *g_h2d_counter += (int64_t)(sizeof(T) * v.size());
    cudaError_t e = b.ensure(sizeof(T) * v.size());
    if (e != cudaSuccess || v.empty()) return e;
    e = cudaMemcpyAsync(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);   // host staging vectors are temporaries
}

}  // namespace

// One mesh on the device: built by vie_set_mesh, read-only afterwards, shared
// by the context and its solve slots (concurrent solves read it together).
struct MeshState {
    bool have_mesh = false;
    vie::Topology topo;
    DevBuf tv, cen, vol, q5, far32, far64, fv, f5, farea, ffar32, ffar64, hf, n32, n64, fn32, fn64, fcen;
    DevBuf mk[4], pr[4], to[4], tdom, tpart;
    DevBuf thalf, tsc[4];   // static integrals of the touching near images (per mesh)
    int npr[4] = {0, 0, 0, 0}, nto[4] = {0, 0, 0, 0};
};

struct vie_ctx {
    int device = 0;
    vie_options opt{};
    std::string err;
    std::shared_ptr<MeshState> mesh = std::make_shared<MeshState>();
    // request (device)
    DevBuf row, coef, wt, kap, ieps, frow, qs, perm, pol, orders, stab, ztab, rtab, ew;
    double z_extent = 0;
    // solve buffers
    DevBuf Z, b, x, r, u, w, V, h, y, Minv, MinvH, amax, tcpack, tcpack2, status, acc, J, rt, cout, xs;
    DevBuf Zh;     // 16-bit copy of Z read by the GMRES products (VIE_FP16 / VIE_BF16)
    size_t ld16 = 0;   // its row stride (column-interleaved layout, vie::ld16)
    // the FP16 block inverses the preconditioner reads (interleaved): offsets and row strides
    std::vector<size_t> moff16, mld16;
    DevBuf dens;   // per-tetrahedron absorbed fractions [2][nt] (request density_out)
    double zh_alpha = 1.0;   // 1 / (power-of-two scale of the FP16 copy)
    // set by the solve server when the request is cancelled: a solve checks it
    // between phases and at every GMRES iteration (the stream is idle there)
    const std::atomic<int> *cancel = nullptr;
    std::vector<double> pinv;   // per domain block: 1 / (power-of-two scale of its FP16 inverse)
    // autotuner choices for this mesh (0: the defaults): the FP32 tables' Ewald
    // split multiplier per incidence class (0 normal, 1 oblique), and the row
    // ranges per resident CTA of the GMRES products; tuned[c]: class c was tuned
    double tune_split[2] = {0.0, 0.0};
    int tune_mv = 0;
    int tune_pivot = 0;   // outer pivot width of the block inversion (0: 512)
    bool tuned[2] = {false, false};
    size_t ld = 0;
    int64_t h2d = 0, d2h = 0;   // bytes copied by the current solve
    // CUDA events for options.timing
    std::vector<cudaEvent_t> events;
    size_t ev_used = 0;
    // solve slots of vie_solve_batch: contexts sharing this mesh, each with its
    // own request and solve buffers and its own stream
    std::vector<std::unique_ptr<vie_ctx>> slots;
    cudaStream_t own_stream = nullptr;
    cudaStream_t aux_stream = nullptr;    // second stream of the block inversion (look-ahead)
    cudaStream_t side_stream = nullptr;   // the smaller domain blocks' inversions and products, beside the largest
    cudaEvent_t side_go = nullptr, side_done = nullptr;
    ~vie_ctx() {
        slots.clear();
        for (auto e : events) cudaEventDestroy(e);
        if (side_go) cudaEventDestroy(side_go);
        if (side_done) cudaEventDestroy(side_done);
        if (own_stream) cudaStreamDestroy(own_stream);
        if (aux_stream) cudaStreamDestroy(aux_stream);
        if (side_stream) cudaStreamDestroy(side_stream);
    }
    cudaEvent_t event() {   // next event of the pool (nullptr when timing is off)
        if (!opt.timing) return nullptr;
        if (ev_used == events.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            events.push_back(e);
        }
        return events[ev_used++];
    }
};

namespace {
double ev_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0;
    if (a && b && cudaEventElapsedTime(&ms, a, b) == cudaSuccess) return ms;
    return 0.0;
}
}  // namespace

namespace {

int fail(vie_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

#define CK(expr)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? VIE_ENOMEM : VIE_ECUDA,        \
                        std::string(#expr) + ": " + cudaGetErrorString(e_));                 \
    } while (0)

struct HostReq {
    double k0, kx, ky, theta;
    std::vector<cplx> eps, kap;          // per domain, exp(j w t) convention
    std::vector<int32_t> perm;           // canonical unknown -> matrix row
    std::vector<int> blk_off, blk_n;     // domain blocks (non-empty)
    vie::EwaldTables ew;
    std::vector<double> orders;          // [n][4]: k_tx, k_ty, k_z, is (0,0)
    double pol[6], kinc[3];
};

int prepare(vie_ctx *ctx, const vie_request *req, HostReq &H) {
    const vie::Topology &T = ctx->mesh->topo;
    if (!(req->lambda_nm > 0) || !std::isfinite(req->lambda_nm)) return fail(ctx, VIE_EINVAL, "lambda must be > 0");
    if (!(std::fabs(req->theta) < M_PI / 2)) return fail(ctx, VIE_EINVAL, "|theta| must be < pi/2");
    H.k0 = 2.0 * M_PI / req->lambda_nm;
    H.theta = req->theta;
    H.kx = H.k0 * std::sin(req->theta) * std::cos(req->phi);
    H.ky = H.k0 * std::sin(req->theta) * std::sin(req->phi);
    H.kinc[0] = H.kx; H.kinc[1] = H.ky; H.kinc[2] = -H.k0 * std::cos(req->theta);
    const double th = req->theta, ph = req->phi;
    const double te[3] = {-std::sin(ph), std::cos(ph), 0.0};
    const double tm[3] = {std::cos(th) * std::cos(ph), std::cos(th) * std::sin(ph), std::sin(th)};
    for (int d = 0; d < 3; ++d) { H.pol[d] = te[d]; H.pol[3 + d] = tm[d]; }
    H.eps.resize(T.n_dom);
    H.kap.resize(T.n_dom);
    for (int d = 0; d < T.n_dom; ++d) {
        cplx e(req->eps[2 * d], -req->eps[2 * d + 1]);   // conjugate: exp(j w t)
        if (!(std::abs(e) > 0) || !std::isfinite(std::abs(e))) return fail(ctx, VIE_EINVAL, "bad permittivity");
        H.eps[d] = e;
        H.kap[d] = 1.0 - 1.0 / e;
    }
    // Eq. (5): the unknowns grouped by material domain into contiguous blocks
    std::vector<double> eps_abs(T.n_dom);
    for (int d = 0; d < T.n_dom; ++d) eps_abs[d] = std::abs(H.eps[d]);
    vie::domain_blocks(T, eps_abs, ctx->opt.precond_block_max, H.perm, H.blk_off, H.blk_n);
    // Ewald parameters and tables (Sec. 2.2) and the propagating Floquet orders
    const char *why = "";
    const bool fp64 = ctx->opt.precision == VIE_FP64;
    const double split = ctx->tune_split[(H.kx == 0.0 && H.ky == 0.0) ? 0 : 1];
    if (int rc = vie::build_ewald_tables(T.a, T.b, H.k0, H.kx, H.ky, ctx->z_extent, fp64, H.ew, &H.orders, &why,
                                         split))
        return fail(ctx, rc, why);
    return VIE_OK;
}

// upload the per-request arrays and build the device views
int upload_request(vie_ctx *ctx, const HostReq &H, vie::DevReq &q, cudaStream_t st) {
    const vie::Topology &T = ctx->mesh->topo;
    std::vector<int32_t> row(4 * (size_t)T.nt);
    std::vector<double> coef(4 * (size_t)T.nt), wt(8 * (size_t)T.nt), kap(2 * (size_t)T.nt), ie(2 * (size_t)T.nt);
    for (int t = 0; t < T.nt; ++t) {
        cplx e = H.eps[T.dom[t]];
        cplx k = H.kap[T.dom[t]];
        kap[2 * t] = k.real(); kap[2 * t + 1] = k.imag();
        cplx iv = 1.0 / e;
        ie[2 * t] = iv.real(); ie[2 * t + 1] = iv.imag();
        for (int i = 0; i < 4; ++i) {
            size_t li = 4 * (size_t)t + i;
            row[li] = H.perm[T.basis[li]];
            coef[li] = T.sgn[li] * T.area[li] / (3.0 * T.vol[t]);
            double sx = T.shift[li] == 1 ? T.a : 0.0, sy = T.shift[li] == 2 ? T.b : 0.0;
            double phs = H.kx * sx + H.ky * sy;
            wt[2 * li] = std::cos(phs);
            wt[2 * li + 1] = std::sin(phs);
        }
    }
    const int nf = (int)T.cf.size();
    std::vector<int32_t> frow(std::max(nf, 1));
    std::vector<double> qs(2 * (size_t)std::max(nf, 1));
    for (int f = 0; f < nf; ++f) {
        int n = T.cf[f];
        frow[f] = H.perm[n];
        cplx kp = H.kap[T.dom[T.tp[n]]];
        cplx km = T.kind[n] == vie::KIND_HALF ? cplx(0, 0) : H.kap[T.dom[T.tm[n]]];
        cplx s = km - kp;
        qs[2 * f] = s.real(); qs[2 * f + 1] = s.imag();
    }
    CK(upload(ctx->row, row, st));
    CK(upload(ctx->coef, coef, st));
    CK(upload(ctx->wt, wt, st));
    CK(upload(ctx->kap, kap, st));
    CK(upload(ctx->ieps, ie, st));
    CK(upload(ctx->frow, frow, st));
    CK(upload(ctx->qs, qs, st));
    CK(upload(ctx->perm, H.perm, st));
    std::vector<double> pol(H.pol, H.pol + 6);
    CK(upload(ctx->pol, pol, st));
    std::vector<double> ord = H.orders;
    if (ord.empty()) ord.assign(4, 0.0);
    CK(upload(ctx->orders, ord, st));
    CK(ctx->ew.ensure(sizeof(vie::EwaldTables)));
    CK(vie::upload_ewald(ctx->ew.as<vie::EwaldTables>(), H.ew, st));
    if (g_h2d_counter) *g_h2d_counter += (int64_t)sizeof(vie::EwaldTables);
    CK(ctx->stab.ensure(sizeof(float) * 4 * vie::NSPAT));
    CK(ctx->ztab.ensure(sizeof(float2) * 4 * vie::NZTAB * std::max(H.ew.n_tab, 1)));
    CK(ctx->rtab.ensure(sizeof(float4) * vie::NZTAB * (2 * (size_t)H.ew.n_tab + 1)));   // real, zero, imaginary
    CK(vie::launch_build_tables(ctx->ew.as<vie::EwaldTables>(), ctx->stab.as<float>(), ctx->ztab.as<float2>(),
                                H.ew.n_tab, st, ctx->rtab.as<float4>()));
    q.stab = ctx->stab.as<float>();
    q.ztab = ctx->ztab.as<float2>();
    q.rtab = ctx->rtab.as<float4>();
    q.ew = ctx->ew.as<vie::EwaldTables>();
    q.ef = vie::make_ewald_f32(H.ew);
    q.k0 = H.k0; q.kx = H.kx; q.ky = H.ky;
    for (int k = 0; k < 9; ++k) {
        const double phs = H.kx * (k / 3 - 1) * ctx->mesh->topo.a + H.ky * (k % 3 - 1) * ctx->mesh->topo.b;
        q.img_ph[2 * k] = std::cos(phs) / (4.0 * M_PI);
        q.img_ph[2 * k + 1] = std::sin(phs) / (4.0 * M_PI);
    }
    for (int d = 0; d < 3; ++d) q.kinc[d] = H.kinc[d];
    for (int d = 0; d < 6; ++d) q.pol[d] = H.pol[d];
    q.row = ctx->row.as<int32_t>();
    q.coef = ctx->coef.as<double>();
    q.wt = ctx->wt.as<double>();
    q.kap = ctx->kap.as<double>();
    q.ieps = ctx->ieps.as<double>();
    q.frow = ctx->frow.as<int32_t>();
    q.qs = ctx->qs.as<double>();
    return VIE_OK;
}

vie::DevMesh dev_mesh(vie_ctx *ctx) {
    const vie::Topology &T = ctx->mesh->topo;
    vie::DevMesh m{};
    m.nt = T.nt; m.N = T.N; m.nf = (int)T.cf.size(); m.nh = (int)T.hf.size();
    m.a = T.a; m.b = T.b;
    m.tv = ctx->mesh->tv.as<double>(); m.cen = ctx->mesh->cen.as<double>(); m.vol = ctx->mesh->vol.as<double>();
    m.q5 = ctx->mesh->q5.as<double>(); m.far32 = ctx->mesh->far32.as<float>(); m.far64 = ctx->mesh->far64.as<double>();
    m.fv = ctx->mesh->fv.as<double>(); m.f5 = ctx->mesh->f5.as<double>(); m.farea = ctx->mesh->farea.as<double>();
    m.ffar32 = ctx->mesh->ffar32.as<float>(); m.ffar64 = ctx->mesh->ffar64.as<double>(); m.hf = ctx->mesh->hf.as<int32_t>();
    m.n32 = ctx->mesh->n32.as<float>(); m.n64 = ctx->mesh->n64.as<double>();
    m.fn32 = ctx->mesh->fn32.as<float>(); m.fn64 = ctx->mesh->fn64.as<double>(); m.fcen = ctx->mesh->fcen.as<double>();
    m.mk_tt = ctx->mesh->mk[0].as<uint16_t>(); m.mk_tf = ctx->mesh->mk[1].as<uint16_t>();
    m.mk_ft = ctx->mesh->mk[2].as<uint16_t>(); m.mk_ff = ctx->mesh->mk[3].as<uint16_t>();
    m.touch_partner = ctx->mesh->tpart.as<int32_t>();
    m.touch_half = ctx->mesh->thalf.as<double>();
    for (int i = 0; i < 4; ++i) m.touch_sc[i] = ctx->mesh->tsc[i].as<double>();
    for (int i = 0; i < 4; ++i) {
        m.pr[i] = ctx->mesh->pr[i].as<vie::NearEntry>();
        m.to[i] = ctx->mesh->to[i].as<vie::NearEntry>();
        m.npr[i] = ctx->mesh->npr[i];
        m.nto[i] = ctx->mesh->nto[i];
    }
    return m;
}

struct Timing {
    cudaEvent_t fill0 = nullptr, fill1 = nullptr, far0 = nullptr, far1 = nullptr, fac0 = nullptr, fac1 = nullptr;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> mv;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pc;   // preconditioner applications
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ot;   // Gram-Schmidt passes
    double pc_bytes = 0;                                   // their algorithmic bytes
    vie::KernelTimer tc;
};

template <typename TZ>
int fill(vie_ctx *ctx, const vie::DevMesh &m, const vie::DevReq &q, bool with_rhs, cudaStream_t st,
         Timing *tm = nullptr) {
    const size_t N = (size_t)ctx->mesh->topo.N;
    ctx->ld = (N + 3) / 4 * 4;
    CK(ctx->Z.ensure(sizeof(TZ) * 2 * ctx->ld * N));
    if (with_rhs) CK(ctx->b.ensure(sizeof(double) * 4 * N));
    const vie::DevMesh &mm = m;
    if (tm && tm->fill0) CK(cudaEventRecord(tm->fill0, st));
    CK(vie::launch_fill<TZ>(mm, q, ctx->Z.as<TZ>(), ctx->ld, with_rhs ? ctx->b.as<double>() : nullptr, st,
                            tm ? tm->far0 : nullptr, tm ? tm->far1 : nullptr));
    if (tm && tm->fill1) CK(cudaEventRecord(tm->fill1, st));
    return VIE_OK;
}

// M^-1 applied block by block: out[blk] = Minv_d in[blk].  The largest block's
// product runs on st, the smaller (latency-bound) ones beside it on the side
// stream, joined before the application returns on st.
template <typename TV>
int precond_apply(vie_ctx *ctx, const HostReq &H, const std::vector<size_t> &moff, const std::vector<size_t> &mld,
                  const TV *in, TV *out, cudaStream_t st) {
    size_t kbig = 0;
    for (size_t k = 1; k < H.blk_n.size(); ++k)
        if (H.blk_n[k] > H.blk_n[kbig]) kbig = k;
    const bool side = H.blk_n.size() > 1 && ctx->side_stream;
    if (side) {
        CK(cudaEventRecord(ctx->side_go, st));
        CK(cudaStreamWaitEvent(ctx->side_stream, ctx->side_go, 0));
    }
    for (size_t k = 0; k < H.blk_off.size(); ++k) {
        const __half *Mi = ctx->MinvH.as<__half>() + 2 * ctx->moff16[k];
        CK((vie::matvec<__half, TV, TV>(Mi, ctx->mld16[k], H.blk_n[k], H.blk_n[k], in + 4 * (size_t)H.blk_off[k],
                                         out + 4 * (size_t)H.blk_off[k], TV(ctx->pinv[k]), false,
                                         side && k != kbig ? ctx->side_stream : st)));
    }
    if (side) {
        CK(cudaEventRecord(ctx->side_done, ctx->side_stream));
        CK(cudaStreamWaitEvent(st, ctx->side_done, 0));
    }
    return VIE_OK;
}

// one application of M^-1 with CUDA events around it (options.timing); the
// algorithmic bytes are one read of every FP16 block inverse plus the vectors
template <typename TV>
int timed_precond(vie_ctx *ctx, const HostReq &H, const std::vector<size_t> &moff, const std::vector<size_t> &mld,
                  const TV *in, TV *out, cudaStream_t st, Timing &tm) {
    cudaEvent_t e0 = ctx->event(), e1 = ctx->event();
    if (e0) CK(cudaEventRecord(e0, st));
    if (int e = precond_apply<TV>(ctx, H, moff, mld, in, out, st)) return e;
    if (e1) {
        CK(cudaEventRecord(e1, st));
        tm.pc.push_back({e0, e1});
        for (size_t k = 0; k < H.blk_n.size(); ++k)
            tm.pc_bytes += 4.0 * (double)H.blk_n[k] * (double)mld[k] + 2.0 * 2 * 2 * sizeof(TV) * H.blk_n[k];
    }
    return VIE_OK;
}

bool cancelled(const vie_ctx *ctx) { return ctx->cancel && ctx->cancel->load(std::memory_order_relaxed) != 0; }

// Default inner-sweep tolerances (options.inner_tol = 0): FP32 products
// 3e-6; the 16-bit copies of Z, rounded to 2^-11 (FP16) or 2^-8 (BF16)
// relative, cannot reduce the FP64 residual of the FP32 Z much further than
// about that in one sweep, so their sweeps stop there and the next refinement
// step continues.
constexpr double INNER_TOL_FP32 = 3e-6;
constexpr double INNER_TOL_FP16 = 1e-3;
constexpr double INNER_TOL_BF16 = 8e-3;

// Left-preconditioned GMRES(m) on diag(A_dd^-1) Z x = diag(A_dd^-1) b for TE
// and TM together (every product reads Z once for both), inside FP64-residual
// iterative refinement: each sweep starts from r = b - Z x formed in FP64 (FP32
// Z: at double length from FP32 arithmetic).  The sweep's products read Z
// itself, or its 16-bit copy ctx->Zh for VIE_FP16 / VIE_BF16.
template <typename TZ, typename TV>
int gmres(vie_ctx *ctx, const HostReq &H, const std::vector<size_t> &moff, const std::vector<size_t> &mld,
          vie_result *res, cudaStream_t st, Timing &tm) {
    const int N = ctx->mesh->topo.N;
    const int m = std::max(2, ctx->opt.restart);
    const bool pre = ctx->opt.use_precond != 0;
    const double tol = ctx->opt.tol;
    const int zin = std::is_same<TV, float>::value ? (ctx->opt.precision == VIE_FP16 ? 1 : ctx->opt.precision == VIE_BF16 ? 2 : 0) : 0;
    const double inner_def = zin == 1 ? INNER_TOL_FP16 : zin == 2 ? INNER_TOL_BF16 : INNER_TOL_FP32;
    const double inner_tol = std::is_same<TV, float>::value
                                 ? std::max(ctx->opt.inner_tol > 0 ? ctx->opt.inner_tol : inner_def, 1e-6)
                                 : tol * 0.1;
    const size_t vs = 4 * (size_t)N;     // stride of one basis vector (two rhs)
    const int mvg = ctx->tune_mv > 0 ? ctx->tune_mv : 1;   // launch shape of the Z products
    CK(ctx->x.ensure(sizeof(double) * vs));
    CK(ctx->r.ensure(sizeof(double) * vs));
    CK(ctx->u.ensure(sizeof(TV) * vs));
    CK(ctx->w.ensure(sizeof(TV) * vs));
    CK(ctx->V.ensure(sizeof(TV) * vs * (m + 1)));
    CK(ctx->h.ensure(sizeof(double) * 4 * (2 * m + 4)));
    CK(ctx->y.ensure(sizeof(double) * 4 * (m + 1)));
    double *x = ctx->x.as<double>(), *r = ctx->r.as<double>(), *hd = ctx->h.as<double>();
    TV *u = ctx->u.as<TV>(), *w = ctx->w.as<TV>(), *V = ctx->V.as<TV>();
    const TZ *Z = ctx->Z.as<TZ>();
    CK(cudaMemsetAsync(x, 0, sizeof(double) * vs, st));
    std::vector<double> hh(4 * (2 * m + 4));
    auto norms2 = [&](const double *vec, double out[2]) -> int {
        CK(vie::dots<double>(vec, 0, 1, vec, N, hd, st));
        CK(cudaMemcpyAsync(hh.data(), hd, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
        ctx->d2h += sizeof(double) * 4;
        CK(cudaStreamSynchronize(st));
        out[0] = std::sqrt(std::max(hh[0], 0.0));
        out[1] = std::sqrt(std::max(hh[2], 0.0));
        return VIE_OK;
    };
    double bn[2];
    if (int e = norms2(ctx->b.as<double>(), bn)) return e;
    const double b_raw[2] = {bn[0], bn[1]};
    for (int p = 0; p < 2; ++p) if (!(bn[p] > 0)) bn[p] = 1.0;
    int iters[2] = {0, 0};
    int total = 0, sweeps = 0;
    double rel[2] = {1, 1};
    bool x_zero = true;   // the first sweep starts from x = 0: r = b
    if (std::is_same<TZ, float>::value) CK(ctx->xs.ensure(sizeof(float) * 8 * (size_t)N));
    while (true) {
        // FP64 residual r = b - Z x (FP32 Z: double-length product from FP32 arithmetic)
        CK(cudaMemcpyAsync(r, ctx->b.p, sizeof(double) * vs, cudaMemcpyDeviceToDevice, st));
        double rn[2] = {b_raw[0], b_raw[1]};
        if (!x_zero) {
            if constexpr (std::is_same<TZ, float>::value)
                CK(vie::matvec_ds(Z, ctx->ld, N, N, x, ctx->xs.as<float>(), r, -1.0, true, st));
            else
                CK((vie::matvec<TZ, double, double>(Z, ctx->ld, N, N, x, r, -1.0, true, st)));
            if (int e = norms2(r, rn)) return e;
        }
        rel[0] = rn[0] / bn[0];
        rel[1] = rn[1] / bn[1];
        bool active[2] = {rel[0] > tol, rel[1] > tol};
        if ((!active[0] && !active[1]) || total >= ctx->opt.max_iter) break;
        ++sweeps;
        // u = r / |r| (per rhs), v0 = M^-1 u
        double s[4] = {rn[0] > 0 ? 1.0 / rn[0] : 0.0, 0.0, rn[1] > 0 ? 1.0 / rn[1] : 0.0, 0.0};
        if (!active[0]) s[0] = 0;
        if (!active[1]) s[2] = 0;
        CK((vie::scale<double, TV>(r, u, N, s, st)));
        if (pre) { if (int e = timed_precond<TV>(ctx, H, moff, mld, u, w, st, tm)) return e; }
        else CK(cudaMemcpyAsync(w, u, sizeof(TV) * vs, cudaMemcpyDeviceToDevice, st));
        CK(vie::dots<TV>(w, 0, 1, w, N, hd, st));
        ctx->d2h += sizeof(double) * 4;
        CK(cudaMemcpyAsync(hh.data(), hd, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        double beta[2] = {std::sqrt(hh[0]), std::sqrt(hh[2])};
        double s0[4] = {beta[0] > 0 ? 1.0 / beta[0] : 0.0, 0, beta[1] > 0 ? 1.0 / beta[1] : 0.0, 0};
        CK((vie::scale<TV, TV>(w, V, N, s0, st)));
        std::vector<cplx> Hm[2], g[2], cs[2], sn[2];
        for (int p = 0; p < 2; ++p) {
            Hm[p].assign((size_t)(m + 1) * m, cplx(0));
            g[p].assign(m + 1, cplx(0));
            cs[p].assign(m, cplx(0));
            sn[p].assign(m, cplx(0));
            g[p][0] = beta[p];
        }
        int kused[2] = {0, 0};
        bool inner_active[2] = {active[0] && beta[0] > 0, active[1] && beta[1] > 0};
        // stop a sweep once the preconditioned residual has dropped by inner_tol,
        // or once it predicts the outer target: the FP64 residual at the end of the
        // sweep is expected near (|g| / beta) |r|, and half of tol |b| is aimed for
        double stop[2];
        for (int p = 0; p < 2; ++p)
            stop[p] = std::max(inner_tol, rn[p] > 0 ? 0.5 * tol * bn[p] / rn[p] : 0.0) * beta[p];
        for (int k = 0; k < m; ++k) {
            if (!inner_active[0] && !inner_active[1]) break;
            TV *vk = V + vs * k;
            TV *vn = V + vs * (k + 1);
            if (cancelled(ctx)) return fail(ctx, VIE_CANCELLED, "cancelled");
            cudaEvent_t e0 = ctx->event(), e1 = ctx->event();
            if (e0) CK(cudaEventRecord(e0, st));
            if constexpr (std::is_same<TV, float>::value) {
                if (zin == 1)
                    CK((vie::matvec<__half, TV, TV>(ctx->Zh.as<__half>(), ctx->ld16, N, N, vk, pre ? u : vn,
                                                    TV(ctx->zh_alpha), false, st, mvg)));
                else if (zin == 2)
                    CK((vie::matvec<__nv_bfloat16, TV, TV>(ctx->Zh.as<__nv_bfloat16>(), ctx->ld16, N, N, vk,
                                                           pre ? u : vn, TV(1), false, st, mvg)));
                else
                    CK((vie::matvec<TZ, TV, TV>(Z, ctx->ld, N, N, vk, pre ? u : vn, TV(1), false, st, mvg)));
            } else {
                CK((vie::matvec<TZ, TV, TV>(Z, ctx->ld, N, N, vk, pre ? u : vn, TV(1), false, st, mvg)));
            }
            if (e1) { CK(cudaEventRecord(e1, st)); tm.mv.push_back({e0, e1}); }
            if (pre) { if (int e = timed_precond<TV>(ctx, H, moff, mld, u, vn, st, tm)) return e; }
            // classical Gram-Schmidt, twice; the projections of both passes and
            // the new norm stay on the device until one copy at the end
            const size_t nh = 4 * (size_t)(k + 1);
            cudaEvent_t o0 = ctx->event(), o1 = ctx->event();
            if (o0) CK(cudaEventRecord(o0, st));
            CK(vie::dots<TV>(V, vs, k + 1, vn, N, hd, st));
            CK(vie::subtract<TV>(V, vs, k + 1, hd, vn, N, st));
            CK(vie::dots<TV>(V, vs, k + 1, vn, N, hd + nh, st));
            CK(vie::subtract<TV>(V, vs, k + 1, hd + nh, vn, N, st));
            CK(vie::dots<TV>(vn, 0, 1, vn, N, hd + 2 * nh, st));
            if (o1) { CK(cudaEventRecord(o1, st)); tm.ot.push_back({o0, o1}); }
            CK(cudaMemcpyAsync(hh.data(), hd, sizeof(double) * (2 * nh + 4), cudaMemcpyDeviceToHost, st));
            ctx->d2h += sizeof(double) * (2 * nh + 4);
            CK(cudaStreamSynchronize(st));
            std::vector<double> hsum(nh);
            for (size_t i = 0; i < nh; ++i) hsum[i] = hh[i] + hh[nh + i];
            double hn[2] = {std::sqrt(std::max(hh[2 * nh], 0.0)), std::sqrt(std::max(hh[2 * nh + 2], 0.0))};
            double sc[4] = {0, 0, 0, 0};
            for (int p = 0; p < 2; ++p) {
                if (!inner_active[p]) continue;
                cplx *Hc = &Hm[p][(size_t)k * (m + 1)];   // column k
                for (int i = 0; i <= k; ++i) Hc[i] = cplx(hsum[4 * i + 2 * p], hsum[4 * i + 2 * p + 1]);
                Hc[k + 1] = hn[p];
                for (int i = 0; i < k; ++i) {   // previous rotations
                    cplx t = std::conj(cs[p][i]) * Hc[i] + std::conj(sn[p][i]) * Hc[i + 1];
                    Hc[i + 1] = -sn[p][i] * Hc[i] + cs[p][i] * Hc[i + 1];
                    Hc[i] = t;
                }
                double den = std::hypot(std::abs(Hc[k]), std::abs(Hc[k + 1]));
                if (den == 0) { cs[p][k] = 1; sn[p][k] = 0; }
                else { cs[p][k] = Hc[k] / den; sn[p][k] = Hc[k + 1] / den; }
                Hc[k] = den;
                Hc[k + 1] = 0;
                g[p][k + 1] = -sn[p][k] * g[p][k];
                g[p][k] = std::conj(cs[p][k]) * g[p][k];
                kused[p] = k + 1;
                ++iters[p];
                if (std::abs(g[p][k + 1]) <= stop[p] || hn[p] <= 1e-300) inner_active[p] = false;
                if (hn[p] > 0) sc[2 * p] = 1.0 / hn[p];
            }
            ++total;
            if (total >= ctx->opt.max_iter) inner_active[0] = inner_active[1] = false;
            CK((vie::scale<TV, TV>(vn, vn, N, sc, st)));
        }
        // y = H^-1 g, x += |r| V y
        int kmax = std::max(kused[0], kused[1]);
        std::vector<double> yv(4 * (size_t)std::max(kmax, 1), 0.0);
        for (int p = 0; p < 2; ++p) {
            int kk = kused[p];
            std::vector<cplx> yy(kk);
            for (int i = kk - 1; i >= 0; --i) {
                cplx sacc = g[p][i];
                for (int j = i + 1; j < kk; ++j) sacc -= Hm[p][(size_t)j * (m + 1) + i] * yy[j];
                yy[i] = sacc / Hm[p][(size_t)i * (m + 1) + i];
            }
            for (int i = 0; i < kk; ++i) {
                cplx v = yy[i] * rn[p];
                yv[4 * i + 2 * p] = v.real();
                yv[4 * i + 2 * p + 1] = v.imag();
            }
        }
        if (kmax > 0) {
            CK(cudaMemcpyAsync(ctx->y.p, yv.data(), sizeof(double) * 4 * kmax, cudaMemcpyHostToDevice, st));
            ctx->h2d += sizeof(double) * 4 * kmax;
            CK(vie::combine<TV>(V, vs, kmax, ctx->y.as<double>(), x, N, st));
            CK(cudaStreamSynchronize(st));
            x_zero = false;
        }
        if (kmax == 0) break;
    }
    res->iterations[0] = iters[0];
    res->iterations[1] = iters[1];
    res->refinements = sweeps;
    res->rel_residual[0] = rel[0];
    res->rel_residual[1] = rel[1];
    return (rel[0] <= tol && rel[1] <= tol) ? VIE_OK : VIE_NOT_CONVERGED;
}

cudaEvent_t pool_event(void *c) { return static_cast<vie_ctx *>(c)->event(); }

template <typename TZ>
int factor(vie_ctx *ctx, const HostReq &H, std::vector<size_t> &moff, std::vector<size_t> &mld, cudaStream_t st,
           vie::KernelTimer *kt) {
    size_t tot = 0;
    moff.clear();
    mld.clear();
    for (size_t k = 0; k < H.blk_n.size(); ++k) {
        size_t l = ((size_t)H.blk_n[k] + 3) / 4 * 4;
        moff.push_back(tot);
        mld.push_back(l);
        tot += l * (size_t)H.blk_n[k];
    }
    CK(ctx->Minv.ensure(sizeof(float) * 2 * std::max<size_t>(tot, 1)));
    CK(ctx->status.ensure(sizeof(int)));
    // the largest block is inverted on st with the look-ahead stream; the others,
    // one after another, on a side stream at the same time (their kernels fill
    // the SMs that the largest block's pivot chain leaves idle)
    size_t kbig = 0;
    for (size_t k = 1; k < H.blk_n.size(); ++k)
        if (H.blk_n[k] > H.blk_n[kbig]) kbig = k;
    size_t pk2 = 1;
    for (size_t k = 0; k < H.blk_n.size(); ++k)
        if (k != kbig) pk2 = std::max(pk2, vie::gj_pack_bytes(H.blk_n[k]));
    CK(ctx->tcpack.ensure(vie::gj_pack_bytes(H.blk_n[kbig])));
    if (H.blk_n.size() > 1) CK(ctx->tcpack2.ensure(pk2));
    if (!ctx->aux_stream) CK(cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking));
    if (!ctx->side_stream) {
        CK(cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ctx->side_go, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ctx->side_done, cudaEventDisableTiming));
    }
    CK(cudaMemsetAsync(ctx->status.p, 0, sizeof(int), st));
    const bool side = H.blk_n.size() > 1;
    if (side) {
        CK(cudaEventRecord(ctx->side_go, st));
        CK(cudaStreamWaitEvent(ctx->side_stream, ctx->side_go, 0));
    }
    for (size_t k = 0; k < H.blk_n.size(); ++k) {
        const bool big = k == kbig;
        cudaStream_t sk = big ? st : ctx->side_stream;
        float *B = ctx->Minv.as<float>() + 2 * moff[k];
        CK((vie::copy_block<TZ, float>(ctx->Z.as<TZ>(), ctx->ld, H.blk_off[k], H.blk_n[k], B, mld[k], sk)));
        CK(vie::gj_invert_tc(B, mld[k], H.blk_n[k], ctx->status.as<int>(), big ? ctx->tcpack.p : ctx->tcpack2.p, sk,
                             big ? ctx->aux_stream : ctx->side_stream, kt,
                             ctx->opt.precond_pivot > 0 ? ctx->opt.precond_pivot
                                                        : (ctx->tune_pivot > 0 ? ctx->tune_pivot : 512)));
    }
    if (side) {
        CK(cudaEventRecord(ctx->side_done, ctx->side_stream));
        CK(cudaStreamWaitEvent(st, ctx->side_done, 0));
    }
    // the applications read FP16 copies of the inverses, each scaled by a power
    // of two that brings its largest entry to [2^13, 2^14) (the scale is undone
    // in the product): half the bytes of every GMRES preconditioner application
    const size_t nblk = H.blk_n.size();
    CK(ctx->amax.ensure(sizeof(unsigned) * std::max<size_t>(nblk, 1)));
    CK(cudaMemsetAsync(ctx->amax.p, 0, sizeof(unsigned) * nblk, st));
    for (size_t k = 0; k < nblk; ++k)
        CK(vie::absmax(ctx->Minv.as<float>() + 2 * moff[k], 2 * mld[k] * (size_t)H.blk_n[k],
                       ctx->amax.as<unsigned>() + k, st));
    int stat = 0;
    std::vector<unsigned> am(nblk);
    ctx->d2h += sizeof(int) + sizeof(unsigned) * nblk;
    CK(cudaMemcpyAsync(&stat, ctx->status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(am.data(), ctx->amax.p, sizeof(unsigned) * nblk, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (stat & 2) return fail(ctx, VIE_DEVICE_TIMEOUT, "a bounded wait of the tensor-core block inversion ran out");
    if (stat) return fail(ctx, VIE_BREAKDOWN, "zero or non-finite pivot while inverting a domain block");
    ctx->moff16.assign(nblk, 0);
    ctx->mld16.assign(nblk, 0);
    size_t tot16 = 0;
    for (size_t k = 0; k < nblk; ++k) {
        ctx->moff16[k] = tot16;
        ctx->mld16[k] = vie::ld16(H.blk_n[k]);
        tot16 += ctx->mld16[k] * (size_t)H.blk_n[k];
    }
    CK(ctx->MinvH.ensure(sizeof(__half) * 2 * std::max<size_t>(tot16, 1)));
    ctx->pinv.assign(nblk, 1.0);
    for (size_t k = 0; k < nblk; ++k) {
        float mx;
        std::memcpy(&mx, &am[k], sizeof(float));
        double scale = 1.0;
        if (mx > 0.f && std::isfinite(mx)) {
            int ex = 0;
            std::frexp((double)mx, &ex);   // mx in [2^(ex-1), 2^ex)
            scale = std::ldexp(1.0, 14 - ex);
        } else if (!(mx == 0.f)) {
            return fail(ctx, VIE_BREAKDOWN, "non-finite entry in a domain block inverse");
        }
        ctx->pinv[k] = 1.0 / scale;
        CK(vie::to_half_il(ctx->Minv.as<float>() + 2 * moff[k], mld[k], H.blk_n[k], H.blk_n[k], (float)scale,
                           ctx->MinvH.as<__half>() + 2 * ctx->moff16[k], st));
    }
    return VIE_OK;
}

// The 16-bit copy of the FP32 Z that the GMRES products read (VIE_FP16:
// scaled by the power of two that brings the largest |Re|, |Im| to
// [2^13, 2^14), undone in the product; VIE_BF16: unscaled)
int make_z16(vie_ctx *ctx, cudaStream_t st) {
    const int N = ctx->mesh->topo.N;
    const size_t count = 2 * ctx->ld * (size_t)N;
    ctx->ld16 = vie::ld16(N);
    CK(ctx->Zh.ensure(sizeof(uint16_t) * 2 * ctx->ld16 * (size_t)N));
    if (ctx->opt.precision == VIE_BF16) {
        ctx->zh_alpha = 1.0;
        CK(vie::to_bf16_il(ctx->Z.as<float>(), ctx->ld, N, N, ctx->Zh.as<__nv_bfloat16>(), st));
        return VIE_OK;
    }
    CK(ctx->amax.ensure(sizeof(unsigned)));
    CK(cudaMemsetAsync(ctx->amax.p, 0, sizeof(unsigned), st));
    CK(vie::absmax(ctx->Z.as<float>(), count, ctx->amax.as<unsigned>(), st));
    unsigned bits = 0;
    CK(cudaMemcpyAsync(&bits, ctx->amax.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    ctx->d2h += sizeof(unsigned);
    CK(cudaStreamSynchronize(st));
    float mx;
    std::memcpy(&mx, &bits, sizeof(float));
    if (!(mx > 0.f) || !std::isfinite(mx)) return fail(ctx, VIE_EINVAL, "impedance matrix is zero or not finite");
    int ex = 0;
    std::frexp((double)mx, &ex);   // mx in [2^(ex-1), 2^ex)
    const double scale = std::ldexp(1.0, 14 - ex);
    ctx->zh_alpha = 1.0 / scale;
    CK(vie::to_half_il(ctx->Z.as<float>(), ctx->ld, N, N, (float)scale, ctx->Zh.as<__half>(), st));
    return VIE_OK;
}

template <typename TZ, typename TV>
int solve_impl(vie_ctx *ctx, const vie_request *req, vie_result *res, cudaStream_t st) {
    using clk = std::chrono::steady_clock;
    HostReq H;
    if (int e = prepare(ctx, req, H)) return e;
    vie::DevMesh m = dev_mesh(ctx);
    vie::DevReq q{};
    const int64_t launches0 = vie::g_launches;
    ctx->h2d = 0;
    ctx->d2h = 0;
    g_h2d_counter = &ctx->h2d;
    int ur = upload_request(ctx, H, q, st);
    g_h2d_counter = nullptr;
    if (ur) return ur;
    ctx->ev_used = 0;
    Timing tm;
    tm.fill0 = ctx->event(); tm.fill1 = ctx->event(); tm.far0 = ctx->event(); tm.far1 = ctx->event();
    tm.fac0 = ctx->event(); tm.fac1 = ctx->event();
    auto t0 = clk::now();
    if (int e = fill<TZ>(ctx, m, q, true, st, &tm)) return e;
    if constexpr (std::is_same<TZ, float>::value) {
        if (ctx->opt.precision == VIE_FP16 || ctx->opt.precision == VIE_BF16)
            if (int e = make_z16(ctx, st)) return e;
    }
    CK(cudaStreamSynchronize(st));
    auto t1 = clk::now();
    if (cancelled(ctx)) return fail(ctx, VIE_CANCELLED, "cancelled");
    std::vector<size_t> moff, mld;
    if (ctx->opt.use_precond) {
        if (tm.fac0) CK(cudaEventRecord(tm.fac0, st));
        if (ctx->opt.timing) { tm.tc.alloc = pool_event; tm.tc.pool = ctx; }
        if (int e = factor<TZ>(ctx, H, moff, mld, st, ctx->opt.timing ? &tm.tc : nullptr)) return e;
        if (tm.fac1) { CK(cudaEventRecord(tm.fac1, st)); CK(cudaStreamSynchronize(st)); }
    }
    auto t2 = clk::now();
    if (cancelled(ctx)) return fail(ctx, VIE_CANCELLED, "cancelled");
    int stat = gmres<TZ, TV>(ctx, H, moff, mld, res, st, tm);
    if (stat < 0) return stat;
    auto t3 = clk::now();
    // post-processing
    const int nd = ctx->mesh->topo.n_dom;
    const int n_orders = (int)H.orders.size() / 4;
    CK(ctx->acc.ensure(sizeof(double) * 2 * nd));
    CK(ctx->J.ensure(sizeof(double) * 24 * std::max(n_orders, 1)));
    CK(ctx->rt.ensure(sizeof(double) * 4));
    const double norm = H.k0 / (ctx->mesh->topo.a * ctx->mesh->topo.b * std::cos(H.theta));
    const int ntet = ctx->mesh->topo.nt;
    double *dens = nullptr;   // per-tetrahedron absorbed fractions [2][nt]
    if (req->density_out) {
        if (req->density_on_device) {
            dens = req->density_out;
        } else {
            CK(ctx->dens.ensure(sizeof(double) * 2 * (size_t)ntet));
            dens = ctx->dens.as<double>();
        }
    }
    CK(vie::launch_post(m, q, ctx->x.as<double>(), ctx->mesh->tdom.as<int32_t>(), nd, norm, ctx->orders.as<double>(),
                        n_orders, ctx->mesh->topo.a, ctx->mesh->topo.b, H.k0 * std::cos(H.theta), ctx->pol.as<double>(),
                        ctx->acc.as<double>(), ctx->J.as<double>(), ctx->rt.as<double>(), dens, st));
    if (req->density_out && !req->density_on_device) {
        CK(cudaMemcpyAsync(req->density_out, dens, sizeof(double) * 2 * (size_t)ntet, cudaMemcpyDeviceToHost, st));
        ctx->d2h += sizeof(double) * 2 * (size_t)ntet;
    }
    std::vector<double> acc(2 * nd), rt(4);
    CK(cudaMemcpyAsync(acc.data(), ctx->acc.p, sizeof(double) * 2 * nd, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(rt.data(), ctx->rt.p, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
    ctx->d2h += sizeof(double) * (2 * nd + 4);
    if (req->coeffs_out) {
        const size_t bytes = sizeof(double) * 4 * (size_t)ctx->mesh->topo.N;
        if (req->coeffs_on_device) {
            CK(vie::launch_unpermute(ctx->x.as<double>(), ctx->perm.as<int32_t>(), ctx->mesh->topo.N, req->coeffs_out, st));
        } else {
            CK(ctx->cout.ensure(bytes));
            CK(vie::launch_unpermute(ctx->x.as<double>(), ctx->perm.as<int32_t>(), ctx->mesh->topo.N, ctx->cout.as<double>(), st));
            CK(cudaMemcpyAsync(req->coeffs_out, ctx->cout.p, bytes, cudaMemcpyDeviceToHost, st));
            ctx->d2h += bytes;
        }
    }
    CK(cudaStreamSynchronize(st));
    auto t4 = clk::now();
    for (int p = 0; p < 2; ++p) {
        for (int d = 0; d < nd; ++d) res->absorbed[p][d] = acc[p * nd + d];
        res->reflectance[p] = rt[2 * p];
        res->transmittance[p] = rt[2 * p + 1];
    }
    auto ms = [](clk::time_point a, clk::time_point b) { return std::chrono::duration<double, std::milli>(b - a).count(); };
    res->t_fill_ms = ms(t0, t1);
    res->t_factor_ms = ms(t1, t2);
    res->t_solve_ms = ms(t2, t3);
    res->t_post_ms = ms(t3, t4);
    res->n_unknowns = ctx->mesh->topo.N;
    res->n_near_pairs = (int32_t)ctx->mesh->topo.near_tt.size();
    res->h2d_bytes = ctx->h2d;
    res->d2h_bytes = ctx->d2h;
    res->far_pair_evals = 16 * (int64_t)ctx->mesh->topo.nt * ctx->mesh->topo.nt;
    res->n_launches = (int32_t)(vie::g_launches - launches0);
    if (ctx->opt.timing) {
        res->k_far_tt_ms = ev_ms(tm.far0, tm.far1);
        res->k_fill_ms = ev_ms(tm.fill0, tm.fill1);
        res->k_factor_ms = ev_ms(tm.fac0, tm.fac1);
        double s = 0;
        for (auto &p : tm.mv) s += ev_ms(p.first, p.second);
        res->k_matvec_ms = s;
        res->k_matvec_n = (int32_t)tm.mv.size();
        double ts = 0, tb = 0, tf = 0;
        for (size_t i = 0; i < tm.tc.ev.size(); ++i) {
            ts += ev_ms(tm.tc.ev[i].first, tm.tc.ev[i].second);
            tb += tm.tc.work[i];
            tf += tm.tc.flops[i];
        }
        res->k_tc_flops = tf;
        res->k_tc_ms = ts;
        res->k_tc_bytes = tb;
        res->k_tc_n = (int32_t)tm.tc.ev.size();
        double sp = 0;
        for (auto &p : tm.pc) sp += ev_ms(p.first, p.second);
        res->k_precond_ms = sp;
        res->k_precond_bytes = tm.pc_bytes;
        res->k_precond_n = (int32_t)tm.pc.size();
        double so = 0;
        for (auto &p : tm.ot) so += ev_ms(p.first, p.second);
        res->k_ortho_ms = so;
    }
    res->status = stat;
    return stat;
}

// Device bytes one solve slot holds for request `req` on the current mesh:
// Z, the block inverses, the Krylov basis and vectors, the touching scratch.
int slot_footprint(vie_ctx *ctx, const vie_request *req, size_t *bytes) {
    HostReq H;
    if (int e = prepare(ctx, req, H)) return e;
    const size_t N = (size_t)ctx->mesh->topo.N, ld = (N + 3) / 4 * 4;
    const bool fp64 = ctx->opt.precision == VIE_FP64;
    const size_t sz = fp64 ? 8 : 4;
    size_t minv = 0, pk1 = 0, pk2 = 0;   // block inverses; packing scratch of the largest block and of the others
    for (int n : H.blk_n) {
        minv += 8 * (((size_t)n + 3) / 4 * 4) * (size_t)n + 4 * vie::ld16(n) * (size_t)n;   // FP32 and FP16 copies
        const size_t pk = vie::gj_pack_bytes(n);
        if (pk > pk1) { pk2 = pk1; pk1 = pk; } else if (pk > pk2) pk2 = pk;
    }
    minv += pk1 + pk2;
    const size_t m = (size_t)std::max(2, ctx->opt.restart);
    const size_t vs = 4 * N;
    size_t b = 2 * sz * ld * N + minv + sz * vs * (m + 3) + 8 * vs * 4 + 64 * (size_t)ctx->mesh->nto[0];
    if (ctx->opt.precision == VIE_FP16 || ctx->opt.precision == VIE_BF16) b += 2 * 2 * vie::ld16((int)N) * N;   // 16-bit copy of Z
    b += (size_t)ctx->mesh->topo.nt * 4 * 64 + (16u << 20);   // request arrays, tables, small buffers
    *bytes = b;
    return VIE_OK;
}

void default_opts(vie_options *o) {
    o->precision = VIE_FP32;
    o->use_precond = 1;
    o->restart = 100;
    o->max_iter = 1000;
    o->tol = 1e-6;
    o->inner_tol = 0;   // per precision (3e-6 FP32, 1e-3 FP16, 8e-3 BF16)
    o->timing = 0;
    o->precond_block_max = 0;
    o->precond_pivot = 0;
    o->autotune = 0;
}

}  // namespace

// quadrature weights and Faddeeva coefficients: uploaded once per device, so
// that creating a context never writes constant memory that running solves read
cudaError_t vie::upload_device_constants(int device) {
    static std::mutex mu;
    static std::vector<char> done;
    std::lock_guard<std::mutex> lock(mu);
    if ((size_t)device < done.size() && done[device]) return cudaSuccess;
    cudaError_t e = vie::upload_constants();
    if (e == cudaSuccess) e = vie::upload_post_constants();
    if (e != cudaSuccess) return e;
    if (done.size() <= (size_t)device) done.resize(device + 1, 0);
    done[device] = 1;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Autotuner: the fill schedule (the FP32 tables' Ewald split multiplier, which
// moves work between the lattice images and the Floquet orders) per incidence
// class, and the launch shape of the GMRES products (row ranges per resident
// CTA), each timed with CUDA events on the caller's mesh and request; the
// fastest is kept in the context for the mesh.
// ---------------------------------------------------------------------------
namespace {
constexpr double TUNE_SPLIT_NORMAL[3] = {1.25, 1.5, 1.75};
constexpr double TUNE_SPLIT_OBLIQUE[3] = {1.0, 1.25, 1.5};
constexpr int TUNE_MV[3] = {1, 2, 4};

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

int incidence_class(const vie_request *req) { return std::sin(req->theta) == 0.0 ? 0 : 1; }

template <typename TZ, typename TV>
int tune_impl(vie_ctx *ctx, const vie_request *req, vie_tune_report *out, cudaStream_t st) {
    using clk = std::chrono::steady_clock;
    const auto w0 = clk::now();
    const int cls = incidence_class(req);
    vie_tune_report r{};
    r.incidence_class = cls;
    EventPair ev;
    CK(cudaEventCreate(&ev.a));
    CK(cudaEventCreate(&ev.b));
    auto elapsed = [&](double &ms) -> int {
        float f = 0.f;
        CK(cudaEventSynchronize(ev.b));
        CK(cudaEventElapsedTime(&f, ev.a, ev.b));
        ms = f;
        return VIE_OK;
    };
    const vie::DevMesh m = dev_mesh(ctx);
    const bool fp32 = ctx->opt.precision != VIE_FP64;
    const double keep = ctx->tune_split[cls];
    double best = 1e300, best_split = 0.0;
    HostReq Hk;   // the request as the last filled candidate prepared it (block structure)
    const int n_split = fp32 ? 3 : 1;   // FP64: the series' own split, one fill for the product timing
    for (int c = 0; c < n_split; ++c) {
        const double cand = fp32 ? (cls == 0 ? TUNE_SPLIT_NORMAL[c] : TUNE_SPLIT_OBLIQUE[c]) : 0.0;
        ctx->tune_split[cls] = cand;
        HostReq H;
        vie::DevReq q{};
        int e = prepare(ctx, req, H);
        if (e == VIE_OK) e = upload_request(ctx, H, q, st);
        if (e != VIE_OK) {
            // a candidate whose tables do not fit is skipped; an error of the
            // request itself fails every candidate and is returned
            if (fp32) { r.split[c] = cand; r.fill_ms[c] = -1.0; }
            if (c + 1 == n_split && best_split == 0.0 && fp32) { ctx->tune_split[cls] = keep; return e; }
            if (!fp32) { ctx->tune_split[cls] = keep; return e; }
            continue;
        }
        Hk = H;
        double ms = 1e300;
        for (int rep = 0; rep < 2; ++rep) {
            CK(cudaEventRecord(ev.a, st));
            if (int fe = fill<TZ>(ctx, m, q, false, st)) { ctx->tune_split[cls] = keep; return fe; }
            CK(cudaEventRecord(ev.b, st));
            double t;
            if (int te = elapsed(t)) return te;
            ms = std::min(ms, t);
        }
        if (fp32) {
            r.split[c] = cand;
            r.fill_ms[c] = ms;
            ++r.n_split;
            if (ms < best) { best = ms; best_split = cand; }
        }
    }
    ctx->tune_split[cls] = fp32 ? best_split : keep;
    r.split_chosen = fp32 ? best_split : 0.0;
    // the GMRES products on the matrix they read (FP16 / BF16: the 16-bit copy)
    const int N = ctx->mesh->topo.N;
    if constexpr (std::is_same<TZ, float>::value) {
        if (ctx->opt.precision == VIE_FP16 || ctx->opt.precision == VIE_BF16)
            if (int e = make_z16(ctx, st)) return e;
    }
    DevBuf xv, yv;
    CK(xv.ensure(sizeof(TV) * 4 * (size_t)N));
    CK(yv.ensure(sizeof(TV) * 4 * (size_t)N));
    CK(cudaMemsetAsync(xv.p, 0, sizeof(TV) * 4 * (size_t)N, st));
    auto product = [&](int g) -> cudaError_t {
        if constexpr (std::is_same<TV, float>::value) {
            if (ctx->opt.precision == VIE_FP16)
                return vie::matvec<__half, TV, TV>(ctx->Zh.as<__half>(), ctx->ld16, N, N, xv.as<TV>(), yv.as<TV>(),
                                                   TV(ctx->zh_alpha), false, st, g);
            if (ctx->opt.precision == VIE_BF16)
                return vie::matvec<__nv_bfloat16, TV, TV>(ctx->Zh.as<__nv_bfloat16>(), ctx->ld16, N, N, xv.as<TV>(),
                                                          yv.as<TV>(), TV(1), false, st, g);
        }
        return vie::matvec<TZ, TV, TV>(ctx->Z.as<TZ>(), ctx->ld, N, N, xv.as<TV>(), yv.as<TV>(), TV(1), false, st, g);
    };
    double bmv = 1e300;
    int bg = 1;
    for (int c = 0; c < 3; ++c) {
        const int g = TUNE_MV[c];
        CK(product(g));   // warm-up
        CK(cudaEventRecord(ev.a, st));
        for (int rep = 0; rep < 5; ++rep) CK(product(g));
        CK(cudaEventRecord(ev.b, st));
        double t;
        if (int te = elapsed(t)) return te;
        r.mv_grid[c] = g;
        r.mv_ms[c] = t / 5.0;
        if (t < bmv) { bmv = t; bg = g; }
    }
    r.n_mv = 3;
    r.mv_chosen = bg;
    ctx->tune_mv = bg;
    // the block inversion's outer pivot width (a property of the mesh's blocks:
    // tuned once per mesh, only where a block is wider than the larger width)
    int nbig = 0;
    for (int nb : Hk.blk_n) nbig = std::max(nbig, nb);
    if (ctx->opt.use_precond && ctx->opt.precond_pivot == 0 && ctx->tune_pivot == 0 && nbig > 1024) {
        const int cand[2] = {512, 1024};
        double bf = 1e300;
        int bp = 512;
        for (int c = 0; c < 2; ++c) {
            ctx->tune_pivot = cand[c];
            std::vector<size_t> moff, mld;
            double ms = 1e300;
            for (int rep = 0; rep < 2; ++rep) {
                CK(cudaEventRecord(ev.a, st));
                if (int fe = factor<TZ>(ctx, Hk, moff, mld, st, nullptr)) { ctx->tune_pivot = 0; return fe; }
                CK(cudaEventRecord(ev.b, st));
                double t;
                if (int te = elapsed(t)) return te;
                ms = std::min(ms, t);
            }
            r.pivot[c] = cand[c];
            r.factor_ms[c] = ms;
            if (ms < bf) { bf = ms; bp = cand[c]; }
        }
        r.n_pivot = 2;
        ctx->tune_pivot = bp;
    }
    r.pivot_chosen = ctx->opt.precond_pivot > 0 ? ctx->opt.precond_pivot : (ctx->tune_pivot > 0 ? ctx->tune_pivot : 512);
    ctx->tuned[cls] = true;
    r.tune_ms = std::chrono::duration<double, std::milli>(clk::now() - w0).count();
    if (out) *out = r;
    return VIE_OK;
}
}  // namespace

extern "C" {

void vie_default_options(vie_options *opt) {
    if (opt) default_opts(opt);
}

int vie_create(vie_ctx **out, int device, const vie_options *opt) {
    if (!out) return VIE_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return VIE_ECUDA;
    vie_ctx *ctx = new (std::nothrow) vie_ctx();
    if (!ctx) return VIE_ENOMEM;
    ctx->device = device;
    default_opts(&ctx->opt);
    if (opt) ctx->opt = *opt;
    if (ctx->opt.precision < VIE_FP64 || ctx->opt.precision > VIE_BF16) { delete ctx; return VIE_EINVAL; }
    if (ctx->opt.precond_pivot != 0 && ctx->opt.precond_pivot != 512 && ctx->opt.precond_pivot != 1024) {
        delete ctx;
        return VIE_EINVAL;
    }
    if (cudaSetDevice(device) != cudaSuccess) { delete ctx; return VIE_ECUDA; }
    if (vie::upload_device_constants(device) != cudaSuccess) {
        delete ctx;
        return VIE_ECUDA;
    }
    *out = ctx;
    return VIE_OK;
}

int vie_set_options(vie_ctx *ctx, const vie_options *opt) {
    if (!ctx || !opt) return VIE_EINVAL;
    if (opt->precision < VIE_FP64 || opt->precision > VIE_BF16) return fail(ctx, VIE_EINVAL, "unknown precision");
    if (opt->restart < 2 || opt->max_iter < 1 || !(opt->tol > 0) || opt->precond_block_max < 0 ||
        !(opt->inner_tol >= 0) || (opt->precond_pivot != 0 && opt->precond_pivot != 512 && opt->precond_pivot != 1024))
        return fail(ctx, VIE_EINVAL, "bad solver options");
    ctx->opt = *opt;
    return VIE_OK;
}

int vie_set_mesh(vie_ctx *ctx, const double *verts, int32_t n_verts, const int32_t *tets, int32_t n_tets,
                 const int32_t *tet_domain, int32_t n_domains, double period_a, double period_b,
                 int32_t active_domain) {
    if (!ctx || !verts || !tets || !tet_domain) return VIE_EINVAL;
    if (n_domains < 1 || n_domains > VIE_MAX_DOMAINS) return fail(ctx, VIE_EINVAL, "n_domains out of range");
    if (active_domain < 0 || active_domain >= n_domains) return fail(ctx, VIE_EINVAL, "active_domain out of range");
    cudaSetDevice(ctx->device);
    // a new mesh object: solve slots still holding the previous one keep it alive
    ctx->mesh = std::make_shared<MeshState>();
    ctx->tune_split[0] = ctx->tune_split[1] = 0.0;   // tuned choices belong to a mesh
    ctx->tune_mv = 0;
    ctx->tune_pivot = 0;
    ctx->tuned[0] = ctx->tuned[1] = false;
    std::string e = vie::build_topology(verts, n_verts, tets, n_tets, tet_domain, n_domains, period_a, period_b,
                                        active_domain, ctx->mesh->topo);
    if (!e.empty()) return fail(ctx, e.find("range") != std::string::npos ? VIE_EINVAL : VIE_BAD_MESH, e);
    const vie::Topology &T = ctx->mesh->topo;
    cudaStream_t st = 0;
    {
        double zlo = 1e300, zhi = -1e300;
        for (int v = 0; v < n_verts; ++v) { zlo = std::min(zlo, verts[3 * v + 2]); zhi = std::max(zhi, verts[3 * v + 2]); }
        ctx->z_extent = zhi - zlo;
    }
    // quadrature points
    double b2[4][4], w2[4], b5[14][4], w5[14], c2[3][3], cw2[3], c5[7][3], cw5[7];
    vie::tet_rule2(b2, w2);
    vie::tet_rule5(b5, w5);
    vie::tri_rule2(c2, cw2);
    vie::tri_rule5(c5, cw5);
    std::vector<double> q5(42 * (size_t)T.nt), far64(28 * (size_t)T.nt);
    for (int t = 0; t < T.nt; ++t) {
        const double *P = &T.tv[12 * (size_t)t];
        for (int k = 0; k < 14; ++k)
            for (int d = 0; d < 3; ++d) {
                double s = 0;
                for (int j = 0; j < 4; ++j) s += b5[k][j] * P[3 * j + d];
                q5[42 * (size_t)t + 3 * k + d] = s;
            }
        double *F = &far64[28 * (size_t)t];
        for (int k = 0; k < 4; ++k)
            for (int d = 0; d < 3; ++d) {
                double s = 0;
                for (int j = 0; j < 4; ++j) s += b2[k][j] * P[3 * j + d];
                F[3 * k + d] = s;
            }
        for (int d = 0; d < 3; ++d) F[12 + d] = T.cen[3 * t + d];
        for (int i = 0; i < 4; ++i)
            for (int d = 0; d < 3; ++d) F[15 + 3 * i + d] = P[3 * i + d] - T.cen[3 * t + d];
        F[27] = T.vol[t] * 0.25;
    }
    std::vector<float> far32(far64.begin(), far64.end());
    std::vector<double> n64(56 * (size_t)T.nt);
    for (int t = 0; t < T.nt; ++t)
        for (int k = 0; k < 14; ++k) {
            for (int d = 0; d < 3; ++d) n64[56 * (size_t)t + 4 * k + d] = q5[42 * (size_t)t + 3 * k + d] - T.cen[3 * t + d];
            n64[56 * (size_t)t + 4 * k + 3] = T.vol[t] * w5[k];
        }
    std::vector<float> n32(n64.begin(), n64.end());
    const int nf = (int)T.cf.size();
    std::vector<double> f5(21 * (size_t)std::max(nf, 1)), ffar64(12 * (size_t)std::max(nf, 1), 0.0),
        farea(std::max(nf, 1));
    for (int f = 0; f < nf; ++f) {
        const double *P = &T.fv[9 * (size_t)f];
        double e1[3] = {P[3] - P[0], P[4] - P[1], P[5] - P[2]}, e2[3] = {P[6] - P[0], P[7] - P[1], P[8] - P[2]};
        double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double A = 0.5 * std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        farea[f] = A;
        for (int k = 0; k < 7; ++k)
            for (int d = 0; d < 3; ++d) {
                double s = 0;
                for (int j = 0; j < 3; ++j) s += c5[k][j] * P[3 * j + d];
                f5[21 * (size_t)f + 3 * k + d] = s;
            }
        for (int k = 0; k < 3; ++k)
            for (int d = 0; d < 3; ++d) {
                double s = 0;
                for (int j = 0; j < 3; ++j) s += c2[k][j] * P[3 * j + d];
                ffar64[12 * (size_t)f + 3 * k + d] = s;
            }
        ffar64[12 * (size_t)f + 9] = A / 3.0;
    }
    std::vector<float> ffar32(ffar64.begin(), ffar64.end());
    std::vector<double> fn64(28 * (size_t)std::max(nf, 1), 0.0), fcen(3 * (size_t)std::max(nf, 1), 0.0);
    for (int f = 0; f < nf; ++f) {
        for (int d = 0; d < 3; ++d) fcen[3 * f + d] = T.fcen[3 * f + d];
        for (int k = 0; k < 7; ++k) {
            for (int d = 0; d < 3; ++d) fn64[28 * (size_t)f + 4 * k + d] = f5[21 * (size_t)f + 3 * k + d] - T.fcen[3 * f + d];
            fn64[28 * (size_t)f + 4 * k + 3] = farea[f] * cw5[k];
        }
    }
    std::vector<float> fn32(fn64.begin(), fn64.end());
    const int nh = (int)T.hf.size();
    // dense near-image masks and the (pair, image) entry lists
    auto masks = [](const std::vector<vie::NearPair> &L, size_t nx, size_t ny) {
        std::vector<uint16_t> mk(std::max<size_t>(nx * ny, 1), 0);
        for (auto &p : L) mk[(size_t)p.x * ny + p.y] = p.mask;
        return mk;
    };
    auto entries = [](const std::vector<vie::NearPair> &L, bool touching) {
        std::vector<vie::NearEntry> out;
        for (auto &p : L)
            for (int k = 0; k < 9; ++k)
                if (((p.mask >> k) & 1u) && (((p.touch >> k) & 1u) != 0) == touching) out.push_back({p.x, p.y, k, 0});
        return out;
    };
    std::vector<int32_t> hf = T.hf;
    if (hf.empty()) hf.push_back(0);
    std::vector<double> fv = T.fv;
    if (fv.empty()) fv.assign(9, 0.0);
    CK(upload(ctx->mesh->tv, T.tv, st));
    CK(upload(ctx->mesh->cen, T.cen, st));
    CK(upload(ctx->mesh->vol, T.vol, st));
    CK(upload(ctx->mesh->q5, q5, st));
    CK(upload(ctx->mesh->far64, far64, st));
    CK(upload(ctx->mesh->far32, far32, st));
    CK(upload(ctx->mesh->fv, fv, st));
    CK(upload(ctx->mesh->f5, f5, st));
    CK(upload(ctx->mesh->farea, farea, st));
    CK(upload(ctx->mesh->ffar64, ffar64, st));
    CK(upload(ctx->mesh->ffar32, ffar32, st));
    CK(upload(ctx->mesh->hf, hf, st));
    CK(upload(ctx->mesh->n64, n64, st));
    CK(upload(ctx->mesh->n32, n32, st));
    CK(upload(ctx->mesh->fn64, fn64, st));
    CK(upload(ctx->mesh->fn32, fn32, st));
    CK(upload(ctx->mesh->fcen, fcen, st));
    CK(upload(ctx->mesh->tdom, T.dom, st));
    const std::vector<vie::NearPair> *lists[4] = {&T.near_tt, &T.near_tf, &T.near_ft, &T.near_ff};
    const size_t dims[4][2] = {{(size_t)T.nt, (size_t)T.nt}, {(size_t)T.nt, (size_t)nf}, {(size_t)nh, (size_t)T.nt},
                               {(size_t)nh, (size_t)nf}};
    for (int i = 0; i < 4; ++i) {
        CK(upload(ctx->mesh->mk[i], masks(*lists[i], dims[i][0], dims[i][1]), st));
        auto p = entries(*lists[i], false), q = entries(*lists[i], true);
        ctx->mesh->npr[i] = (int)p.size();
        ctx->mesh->nto[i] = (int)q.size();
        if (p.empty()) p.push_back({0, 0, 0, 0});
        if (q.empty()) q.push_back({0, 0, 0, 0});
        CK(upload(ctx->mesh->pr[i], p, st));
        CK(upload(ctx->mesh->to[i], q, st));
        if (i == 0) {   // partner (y, x, 8-k) of every touching tetrahedron entry
            std::map<std::tuple<int, int, int>, int> idx;
            for (int e = 0; e < ctx->mesh->nto[0]; ++e) idx[std::make_tuple(q[e].x, q[e].y, q[e].k)] = e;
            std::vector<int32_t> part(std::max(ctx->mesh->nto[0], 1), 0);
            for (int e = 0; e < ctx->mesh->nto[0]; ++e) {
                auto it = idx.find(std::make_tuple(q[e].y, q[e].x, 8 - q[e].k));
                if (it == idx.end()) return fail(ctx, VIE_BAD_MESH, "near-pair lists are not symmetric");
                part[e] = it->second;
            }
            CK(upload(ctx->mesh->tpart, part, st));
        }
    }
    // static integrals of the touching near images: geometry only, once per mesh
    CK(ctx->mesh->thalf.ensure(sizeof(double) * 8 * std::max(ctx->mesh->nto[0], 1)));
    double *tsc[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int i = 1; i < 4; ++i) {
        CK(ctx->mesh->tsc[i].ensure(sizeof(double) * std::max(ctx->mesh->nto[i], 1)));
        tsc[i] = ctx->mesh->tsc[i].as<double>();
    }
    {
        const vie::DevMesh dm = dev_mesh(ctx);
        CK(vie::launch_static_cache(dm, ctx->mesh->thalf.as<double>(), tsc, st));
        CK(cudaStreamSynchronize(st));
    }
    ctx->mesh->have_mesh = true;
    return VIE_OK;
}

int32_t vie_num_unknowns(const vie_ctx *ctx) { return (ctx && ctx->mesh->have_mesh) ? ctx->mesh->topo.N : 0; }

int vie_tune(vie_ctx *ctx, const vie_request *req, vie_tune_report *report, void *stream) {
    if (!ctx || !req) return VIE_EINVAL;
    if (!ctx->mesh->have_mesh) return fail(ctx, VIE_EINVAL, "no mesh set");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    return ctx->opt.precision == VIE_FP64 ? tune_impl<double, double>(ctx, req, report, st)
                                          : tune_impl<float, float>(ctx, req, report, st);
}

int vie_solve(vie_ctx *ctx, const vie_request *req, vie_result *res, void *stream) {
    if (!ctx || !req || !res) return VIE_EINVAL;
    if (!ctx->mesh->have_mesh) return fail(ctx, VIE_EINVAL, "no mesh set");
    std::memset(res, 0, sizeof(*res));
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (ctx->opt.autotune && !ctx->tuned[incidence_class(req)]) {   // first solve of this class on the mesh
        if (int e = vie_tune(ctx, req, nullptr, stream)) { res->status = e; return e; }
    }
    int r = ctx->opt.precision == VIE_FP64 ? solve_impl<double, double>(ctx, req, res, st)
                                           : solve_impl<float, float>(ctx, req, res, st);
    res->status = r;
    return r;
}

int vie_solve_batch(vie_ctx *ctx, const vie_request *reqs, vie_result *res, int32_t n, int32_t max_slots,
                    int32_t *slots_used, void *stream) {
    if (slots_used) *slots_used = 0;
    if (!ctx || (n > 0 && (!reqs || !res)) || n < 0 || max_slots < 1) return VIE_EINVAL;
    if (!ctx->mesh->have_mesh) return fail(ctx, VIE_EINVAL, "no mesh set");
    if (n == 0) return VIE_OK;
    std::memset(res, 0, sizeof(vie_result) * (size_t)n);
    cudaSetDevice(ctx->device);
    // work the caller queued on its stream (for example device coefficient
    // buffers being prepared) completes before any slot starts
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    // admission by HBM footprint: a slot is opened only while its buffers fit
    // in the free device memory (less 5% and 1 GB of headroom)
    // autotune: each incidence class of the batch once, here, before the slots start
    if (ctx->opt.autotune) {
        for (int i = 0; i < n; ++i)
            if (!ctx->tuned[incidence_class(&reqs[i])])
                if (int e = vie_tune(ctx, &reqs[i], nullptr, stream)) return e;
    }
    size_t per = 0;
    if (int e = slot_footprint(ctx, &reqs[0], &per)) return e;
    int want = std::min<int>(max_slots, n);
    std::vector<vie_ctx *> use;
    use.push_back(ctx);
    for (int k = 1; k < want; ++k) {
        if ((size_t)k > ctx->slots.size()) {
            size_t free_b = 0, total_b = 0;
            CK(cudaMemGetInfo(&free_b, &total_b));
            const size_t headroom = total_b / 20 + (1ull << 30);
            if (free_b < headroom || free_b - headroom < per) break;
            std::unique_ptr<vie_ctx> c(new (std::nothrow) vie_ctx());
            if (!c) break;
            c->device = ctx->device;
            CK(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
            ctx->slots.push_back(std::move(c));
        }
        vie_ctx *c = ctx->slots[k - 1].get();
        c->opt = ctx->opt;
        c->mesh = ctx->mesh;
        for (int k2 = 0; k2 < 2; ++k2) { c->tune_split[k2] = ctx->tune_split[k2]; c->tuned[k2] = ctx->tuned[k2]; }
        c->tune_mv = ctx->tune_mv;
        c->tune_pivot = ctx->tune_pivot;
        c->z_extent = ctx->z_extent;
        use.push_back(c);
    }
    if (!ctx->own_stream) CK(cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking));
    if (slots_used) *slots_used = (int32_t)use.size();
    std::atomic<int> next{0};
    auto worker = [&](vie_ctx *c) {
        cudaSetDevice(c->device);
        for (int i = next++; i < n; i = next++) vie_solve(c, &reqs[i], &res[i], c->own_stream);
    };
    std::vector<std::thread> th;
    for (size_t k = 1; k < use.size(); ++k) th.emplace_back(worker, use[k]);
    worker(ctx);
    for (auto &t : th) t.join();
    int worst = VIE_OK;
    for (int i = 0; i < n; ++i)
        if (res[i].status < 0) { worst = res[i].status; break; }
    if (worst < 0) {
        for (vie_ctx *c : use)
            if (!c->err.empty()) { ctx->err = c->err; break; }
        return worst;
    }
    for (int i = 0; i < n; ++i)
        if (res[i].status > 0) return res[i].status;
    return VIE_OK;
}

int vie_fill_matrix(vie_ctx *ctx, const vie_request *req, double *Z_host, double *b_host, void *stream) {
    if (!ctx || !req || !Z_host) return VIE_EINVAL;
    if (!ctx->mesh->have_mesh) return fail(ctx, VIE_EINVAL, "no mesh set");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    vie_options saved = ctx->opt;
    ctx->opt.precision = VIE_FP64;
    HostReq H;
    int e = prepare(ctx, req, H);
    ctx->opt = saved;
    if (e) return e;
    vie::DevMesh m = dev_mesh(ctx);
    vie::DevReq q{};
    if ((e = upload_request(ctx, H, q, st))) return e;
    if ((e = fill<double>(ctx, m, q, true, st))) return e;
    const int N = ctx->mesh->topo.N;
    std::vector<double> Zp((size_t)2 * ctx->ld * N), bp(4 * (size_t)N);
    CK(cudaMemcpyAsync(Zp.data(), ctx->Z.p, sizeof(double) * Zp.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(bp.data(), ctx->b.p, sizeof(double) * bp.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int i = 0; i < N; ++i) {
        size_t ri = H.perm[i];
        for (int j = 0; j < N; ++j) {
            size_t rj = H.perm[j];
            Z_host[2 * ((size_t)i * N + j)] = Zp[2 * (ri * ctx->ld + rj)];
            Z_host[2 * ((size_t)i * N + j) + 1] = Zp[2 * (ri * ctx->ld + rj) + 1];
        }
        if (b_host)
            for (int k = 0; k < 4; ++k) b_host[4 * (size_t)i + k] = bp[4 * ri + k];
    }
    return VIE_OK;
}

int vie_fill_matrix_prec(vie_ctx *ctx, const vie_request *req, double *Z_host, void *stream) {
    if (!ctx || !req || !Z_host) return VIE_EINVAL;
    if (!ctx->mesh->have_mesh) return fail(ctx, VIE_EINVAL, "no mesh set");
    if (ctx->opt.precision == VIE_FP64) return vie_fill_matrix(ctx, req, Z_host, nullptr, stream);
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    HostReq H;
    int e = prepare(ctx, req, H);
    if (e) return e;
    vie::DevMesh m = dev_mesh(ctx);
    vie::DevReq q{};
    if ((e = upload_request(ctx, H, q, st))) return e;
    if ((e = fill<float>(ctx, m, q, false, st))) return e;
    const int N = ctx->mesh->topo.N;
    std::vector<float> Zp((size_t)2 * ctx->ld * N);
    if (ctx->opt.precision == VIE_FP16 || ctx->opt.precision == VIE_BF16) {
        // the 16-bit copy the GMRES products read, widened, its scale undone
        if ((e = make_z16(ctx, st))) return e;
        std::vector<uint16_t> Zb(2 * ctx->ld16 * (size_t)N);
        CK(cudaMemcpyAsync(Zb.data(), ctx->Zh.p, sizeof(uint16_t) * Zb.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        // back from the column-interleaved layout to rows of ld entries
        for (int r = 0; r < N; ++r)
            for (int c = 0; c < N; ++c)
                for (int k = 0; k < 2; ++k) {
                    const uint16_t bits = Zb[2 * ((size_t)r * ctx->ld16 + vie::il_pos((size_t)c)) + k];
                    float v;
                    if (ctx->opt.precision == VIE_FP16) {
                        __half_raw h;
                        h.x = bits;
                        v = (float)((double)__half2float(__half(h)) * ctx->zh_alpha);
                    } else {
                        __nv_bfloat16_raw h;
                        h.x = bits;
                        v = __bfloat162float(__nv_bfloat16(h));
                    }
                    Zp[2 * ((size_t)r * ctx->ld + c) + k] = v;
                }
    } else {
        CK(cudaMemcpyAsync(Zp.data(), ctx->Z.p, sizeof(float) * Zp.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    for (int i = 0; i < N; ++i) {
        size_t ri = H.perm[i];
        for (int j = 0; j < N; ++j) {
            size_t rj = H.perm[j];
            Z_host[2 * ((size_t)i * N + j)] = Zp[2 * (ri * ctx->ld + rj)];
            Z_host[2 * ((size_t)i * N + j) + 1] = Zp[2 * (ri * ctx->ld + rj) + 1];
        }
    }
    return VIE_OK;
}

int vie_domain_block(vie_ctx *ctx, const vie_request *req, int32_t block, int32_t *n_out, int32_t *unknowns,
                     double *Zdd_host, double *Minv_host, void *stream) {
    if (!ctx || !req || !n_out || block < 0) return VIE_EINVAL;
    if (!ctx->mesh->have_mesh) return fail(ctx, VIE_EINVAL, "no mesh set");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    HostReq H;
    int e = prepare(ctx, req, H);
    if (e) return e;
    if (block >= (int)H.blk_n.size()) return fail(ctx, VIE_EINVAL, "block index out of range");
    const int n = H.blk_n[block], off = H.blk_off[block];
    *n_out = n;
    if (!unknowns && !Zdd_host && !Minv_host) return VIE_OK;
    vie::DevMesh m = dev_mesh(ctx);
    vie::DevReq q{};
    if ((e = upload_request(ctx, H, q, st))) return e;
    std::vector<size_t> moff, mld;
    const size_t ldz = ((size_t)ctx->mesh->topo.N + 3) / 4 * 4;
    if (ctx->opt.precision == VIE_FP64) {
        if ((e = fill<double>(ctx, m, q, false, st))) return e;
        if ((e = factor<double>(ctx, H, moff, mld, st, nullptr))) return e;
    } else {
        if ((e = fill<float>(ctx, m, q, false, st))) return e;
        if ((e = factor<float>(ctx, H, moff, mld, st, nullptr))) return e;
    }
    if (unknowns)
        for (int i = 0; i < ctx->mesh->topo.N; ++i)
            if (H.perm[i] >= off && H.perm[i] < off + n) unknowns[H.perm[i] - off] = i;
    if (Zdd_host) {
        const size_t sz = ctx->opt.precision == VIE_FP64 ? 8 : 4;
        std::vector<char> row(2 * sz * (size_t)n);
        for (int i = 0; i < n; ++i) {
            const char *src = static_cast<const char *>(ctx->Z.p) + 2 * sz * ((size_t)(off + i) * ldz + off);
            CK(cudaMemcpyAsync(row.data(), src, row.size(), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            for (size_t k = 0; k < 2 * (size_t)n; ++k)
                Zdd_host[2 * (size_t)i * n + k] = sz == 8 ? reinterpret_cast<const double *>(row.data())[k]
                                                          : reinterpret_cast<const float *>(row.data())[k];
        }
    }
    if (Minv_host) {
        std::vector<float> B(2 * mld[block] * (size_t)n);
        CK(cudaMemcpyAsync(B.data(), ctx->Minv.as<float>() + 2 * moff[block], sizeof(float) * B.size(),
                           cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < 2 * n; ++k) Minv_host[2 * (size_t)i * n + k] = B[2 * (size_t)i * mld[block] + k];
    }
    return VIE_OK;
}

int vie_check_device_wait(int device, int32_t arrive, int32_t polls) {
    if (polls < 1 || polls > 1000000) return VIE_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return VIE_ECUDA;
    int *status = nullptr;
    if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) return VIE_ENOMEM;
    int host = 0, rc = VIE_OK;
    if (cudaMemset(status, 0, sizeof(int)) != cudaSuccess || vie::wait_check(arrive != 0, polls, status, 0) != cudaSuccess ||
        cudaMemcpy(&host, status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = VIE_ECUDA;
    cudaFree(status);
    if (rc != VIE_OK) return rc;
    return (host & 2) ? VIE_DEVICE_TIMEOUT : VIE_OK;
}

int vie_fma_peak(int device, int32_t precision, double *tflops) {
    if (!tflops || (precision != VIE_FP64 && precision != VIE_FP32)) return VIE_EINVAL;
    *tflops = 0;
    if (cudaSetDevice(device) != cudaSuccess) return VIE_ECUDA;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return VIE_ECUDA;
    int rc = VIE_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = VIE_ECUDA;
    // launches of growing length until one runs for at least 100 ms (the short
    // ones warm the clocks up), then three at that length: the best rate counts
    const bool fp64 = precision == VIE_FP64;
    int iters = fp64 ? 16 : 256, timed = 0;
    double best = 0, flops = 0;
    for (int k = 0; rc == VIE_OK && k < 24 && timed < 3; ++k) {
        float ms = 0;
        if (vie::fma_peak(fp64, iters, st, e0, e1, &flops) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = VIE_ECUDA;
            break;
        }
        if (ms < 100.f) { iters *= 2; continue; }
        best = std::max(best, flops / (ms * 1e-3) / 1e12);
        ++timed;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    *tflops = best;
    return rc;
}

int vie_erfcx(vie_ctx *ctx, const double *u, double *out, int32_t n, int32_t precision) {
    if (!ctx || !u || !out || n < 0) return VIE_EINVAL;
    if (n == 0) return VIE_OK;
    cudaSetDevice(ctx->device);
    cudaStream_t st = 0;
    DevBuf du, dout;
    CK(du.ensure(sizeof(double) * 2 * n));
    CK(dout.ensure(sizeof(double) * 2 * n));
    CK(cudaMemcpy(du.p, u, sizeof(double) * 2 * n, cudaMemcpyHostToDevice));
    CK(vie::launch_erfcx(du.as<double>(), dout.as<double>(), n, precision == VIE_FP64, st));
    CK(cudaMemcpy(out, dout.p, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost));
    return VIE_OK;
}

int vie_green(vie_ctx *ctx, const vie_request *req, const double *d, double *out, int32_t n, int32_t precision) {
    if (!ctx || !req || !d || !out || n < 0) return VIE_EINVAL;
    if (!ctx->mesh->have_mesh) return fail(ctx, VIE_EINVAL, "no mesh set (the period comes from the mesh)");
    if (n == 0) return VIE_OK;
    cudaSetDevice(ctx->device);
    vie_options saved = ctx->opt;
    const double saved_z = ctx->z_extent;
    ctx->opt.precision = precision == VIE_FP64 ? VIE_FP64 : VIE_FP32;
    for (int i = 0; i < n; ++i) ctx->z_extent = std::max(ctx->z_extent, std::fabs(d[3 * i + 2]));   // table range
    HostReq H;
    int e = prepare(ctx, req, H);
    ctx->opt = saved;
    ctx->z_extent = saved_z;
    if (e) return e;
    cudaStream_t st = 0;
    CK(ctx->ew.ensure(sizeof(vie::EwaldTables)));
    CK(vie::upload_ewald(ctx->ew.as<vie::EwaldTables>(), H.ew, st));
    CK(ctx->stab.ensure(sizeof(float) * 4 * vie::NSPAT));
    CK(ctx->ztab.ensure(sizeof(float2) * 4 * vie::NZTAB * std::max(H.ew.n_tab, 1)));
    CK(ctx->rtab.ensure(sizeof(float4) * vie::NZTAB * (2 * (size_t)H.ew.n_tab + 1)));   // real, zero, imaginary
    CK(vie::launch_build_tables(ctx->ew.as<vie::EwaldTables>(), ctx->stab.as<float>(), ctx->ztab.as<float2>(),
                                H.ew.n_tab, st, ctx->rtab.as<float4>()));
    DevBuf dd, dout;
    CK(dd.ensure(sizeof(double) * 3 * n));
    CK(dout.ensure(sizeof(double) * 2 * n));
    CK(cudaMemcpy(dd.p, d, sizeof(double) * 3 * n, cudaMemcpyHostToDevice));
    CK(vie::launch_green(dd.as<double>(), dout.as<double>(), n, precision == VIE_FP64, ctx->stab.as<float>(),
                         ctx->ztab.as<float2>(), ctx->ew.as<vie::EwaldTables>(), vie::make_ewald_f32(H.ew), st,
                         ctx->rtab.as<float4>()));
    CK(cudaMemcpy(out, dout.p, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost));
    return VIE_OK;
}

const char *vie_status_str(int s) {
    switch (s) {
        case VIE_OK: return "VIE_OK";
        case VIE_NOT_CONVERGED: return "VIE_NOT_CONVERGED";
        case VIE_PENDING: return "VIE_PENDING";
        case VIE_EINVAL: return "VIE_EINVAL";
        case VIE_ENOMEM: return "VIE_ENOMEM";
        case VIE_ECUDA: return "VIE_ECUDA";
        case VIE_RAYLEIGH_ANOMALY: return "VIE_RAYLEIGH_ANOMALY";
        case VIE_DEVICE_TIMEOUT: return "VIE_DEVICE_TIMEOUT";
        case VIE_BAD_MESH: return "VIE_BAD_MESH";
        case VIE_CANCELLED: return "VIE_CANCELLED";
        case VIE_BREAKDOWN: return "VIE_BREAKDOWN";
        default: return "VIE_UNKNOWN";
    }
}

const char *vie_last_error(const vie_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

void vie_destroy(vie_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    delete ctx;
}

}  // extern "C"

namespace vie {
void set_cancel_flag(vie_ctx *ctx, const std::atomic<int> *flag) {
    if (ctx) ctx->cancel = flag;
}

// Free the device memory of a context: its mesh (unless a solve slot shares
// it), the request arrays and the solve buffers (Z, block inverses, Krylov
// state).  The context stays usable: the next vie_set_mesh and vie_solve
// allocate again.  Used by the solve server to give memory back.
void release_device_memory(vie_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    ctx->slots.clear();
    ctx->mesh = std::make_shared<MeshState>();
    DevBuf *bufs[] = {&ctx->row, &ctx->coef, &ctx->wt, &ctx->kap, &ctx->ieps, &ctx->frow, &ctx->qs,
                      &ctx->perm, &ctx->pol, &ctx->orders, &ctx->stab, &ctx->ztab, &ctx->rtab, &ctx->ew,
                      &ctx->Z, &ctx->b, &ctx->x, &ctx->r, &ctx->u, &ctx->w, &ctx->V, &ctx->h, &ctx->y,
                      &ctx->Minv, &ctx->MinvH, &ctx->amax, &ctx->tcpack, &ctx->tcpack2, &ctx->status, &ctx->acc,
                      &ctx->J, &ctx->xs, &ctx->Zh, &ctx->dens,
                      &ctx->rt, &ctx->cout};
    for (DevBuf *b : bufs) b->release();
}
}  // namespace vie
