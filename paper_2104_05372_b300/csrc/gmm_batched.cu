// Batched GMM objective + gradient (A8): many mixture instances of uneven N, D
// and K in a handful of persistent kernels, meant to be captured once in a CUDA
// graph and replayed.
//
// The host turns the instances into work lists, one per (padded dimension,
// phase): parameter expansion (instance, component), forward (instance,
// 128-point tile), backward Accum (instance, component group, point chunk),
// finalize (instance, component, plus one objective item per instance).
// Forward and backward items are sorted by estimated cost, largest first
// (longest-processing-time order), so that the long items start early and the
// short ones fill the tail. Persistent CTAs pull item indices from an atomic
// counter and run the same per-block bodies as the per-call kernels
// (gmm_kernels.cuh): flattening the nested loops over instances, tiles and
// components into one parallel loop (Sec. 6.1.1).
//
// gmm_batched_prepare writes the descriptors and work lists into the workspace
// (one host-to-device copy, then a stream synchronisation); gmm_batched_vjp only
// enqueues memsets and kernels, so it can be captured in a graph.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "gmm_internal.cuh"
#include "gmm_kernels.cuh"
#include "trace.cuh"

namespace gpa {
namespace {

struct BInst {
    const float *x, *alpha, *mu, *q, *l;
    float *d_alpha, *d_mu, *d_q, *d_l;
    double* out;
    float *rec, *bS, *bM, *lj, *lse;
    double *scal, *lpk, *fwd;
    int64_t n, tiles_per_chunk;
    double gamma, seed, cw;  // cw: gmm_prior_const(d, m, gamma)
    int d, k, m, dp, nchunks, ntiles128;
};

struct BItem {
    int inst, a, b, pad;
};

constexpr int kClasses = 5;  // padded dimension 8, 16, 32, 64, 128
static_assert(kClasses == GPA_BATCH_CLASSES, "classes of gpa_batched_opts");
// phases: prep, forward, backward in default groups, backward in small groups, finalize
constexpr int kPhPrep = 0, kPhFwd = 1, kPhBwd = 2, kPhBwdSmall = 3, kPhFin = 4, kPhases = 5;
int class_of(int dp) { return dp == 8 ? 0 : dp == 16 ? 1 : dp == 32 ? 2 : dp == 64 ? 3 : 4; }
// D <= 8 has a class of its own here (the per-call path pads it to 16)
int batched_dp(int d) { return d <= 8 ? 8 : gmm_dp(d); }

size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

// D <= 8 kernels: 128 points per forward item (one per thread); backward items
// of up to 16 components over 128-point tiles
constexpr int kD8Points = 128, kD8Group = 16, kD8Rec = 8 * 8 + 8 + 4, kD8Stage = 64;

int nblk(int dp) { return (dp / 8) * (dp / 8 + 1) / 2; }
int bwd_tpb(int dp) {
    return dp == 8 ? kD8Points : dp == 16 ? Bwd<16>::TPB : dp == 32 ? Bwd<32>::TPB : dp == 64 ? Bwd<64>::TPB
                                                                                               : Bwd<128>::TPB;
}
int gc_of(int dp) {
    return dp == 8 ? kD8Group : dp == 16 ? Bwd<16>::GC : dp == 32 ? Bwd<32>::GC : dp == 64 ? Bwd<64>::GC
                                                                                           : Bwd<128>::GC;
}
// small component groups (sequential layout): components and threads per CTA
constexpr int kSmallGc16 = 10, kSmallGc32 = 6;
int small_gc_of(int dp) { return dp == 16 ? kSmallGc16 : dp == 32 ? kSmallGc32 : 0; }
int small_threads_of(int dp) {
    return dp == 16 ? Bwd<16, kSmallGc16>::THREADS : dp == 32 ? Bwd<32, kSmallGc32>::THREADS : 0;
}
int bwd_threads_of(int dp) { return dp == 16 ? Bwd<16>::THREADS : dp == 32 ? Bwd<32>::THREADS : 0; }
// the small groups for this instance: fewer thread slots per point over its components
bool use_small_groups(int dp, int k) {
    const int gs = small_gc_of(dp);
    if (gs == 0) return false;
    const int gb = gc_of(dp);
    return (int64_t)((k + gs - 1) / gs) * small_threads_of(dp) < (int64_t)((k + gb - 1) / gb) * bwd_threads_of(dp);
}

// Tensor-core instances of one padded dimension run as a concatenated class
// (gmm_tc_cat_run: one launch per stage over all their tiles) when the
// class's BF16 responsibilities fit kCatRBytes; otherwise each instance runs
// the per-call stages in a workspace region of its own, on the forked streams.
constexpr size_t kCatRBytes = (size_t)8 << 30;
struct CatPlan {
    bool on = false;
    int tdp = 0;
    std::vector<int> members;  // instance indices
    std::vector<TcCatInst> cinst;
    std::vector<int> tile_inst;
    std::vector<int2> fwd_tiles;
    std::vector<int4> gram_items;
    int64_t np = 0, kc = 0, kr = 0;
    size_t off_cinst = 0, off_tile_inst = 0, off_fwd_tiles = 0, off_gram_items = 0;
    size_t off_rec = 0, off_tails = 0, off_xb = 0, off_xl = 0, off_qb = 0, off_ql = 0, off_rb = 0, off_xt = 0,
           off_lse = 0, off_lj = 0;
};

struct Plan {
    std::vector<BInst> inst;
    std::vector<BItem> items[kClasses][kPhases];
    std::vector<int> tc;          // instances on the per-instance tensor-core path
    std::vector<size_t> tc_off;   // their workspace regions (per instance, indexed like tc)
    CatPlan cat[2];               // concatenated tensor-core classes: padded dimension 64, 128
    size_t off_desc, off_items[kClasses][kPhases], off_counters, off_partials, partial_bytes, off_regions;
    size_t total;
};

// Workspace of one tensor-core instance: the per-call layout with the whole
// log-joint resident. Every tensor-core instance has a region of its own, so
// that its parameter expansion and finalize run in the class's persistent
// kernels before and after the contractions (which go one instance per launch).
size_t tc_instance_bytes(const gpa_gmm_instance& I) {
    return gpa_gmm_workspace_bytes(I.n, I.d, I.k, GPA_PREC_BF16_TC, 0);
}

// Tensor-core instances run as separate launches; small ones would leave most
// SMs idle one after another, so they are spread over kTcLanes streams forked
// from (and joined back into) the caller's stream with events: capturable in
// the same CUDA graph. The streams and events are the library's, made once per
// device by gmm_batched_prepare (before any capture) and kept for the process.
constexpr int kTcLanes = 8;
constexpr int kTcMaxDevices = 64;
struct TcLanes {
    cudaStream_t st[kTcLanes];
    cudaEvent_t fork, join[kTcLanes];
    bool ready;
};
TcLanes g_tc_lanes[kTcMaxDevices];
std::mutex g_tc_lanes_mu;

TcLanes* tc_lanes(bool create) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kTcMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_tc_lanes_mu);
    TcLanes& L = g_tc_lanes[dev];
    if (!L.ready && create) {
        bool ok = cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; ok && i < kTcLanes; ++i)
            ok = cudaStreamCreateWithFlags(&L.st[i], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&L.join[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            (void)cudaGetLastError();
            return nullptr;
        }
        L.ready = true;
    }
    return L.ready ? &L : nullptr;
}

// Deterministic plan: workspace offsets are relative (base = 0) until bound.
bool make_plan(const gpa_gmm_instance* in, int n_inst, const gpa_batched_opts& O, char* base, Plan& P) {
    P.inst.resize(n_inst);
    size_t off = 256;  // header
    P.off_desc = off;
    off = a256(off + sizeof(BInst) * (size_t)n_inst);
    // item lists
    for (int i = 0; i < n_inst; ++i) {
        const gpa_gmm_instance& I = in[i];
        if (I.n < 1 || I.d < 1 || I.d > 128 || I.k < 1 || I.k > 4096 || !(I.gamma > 0.0)) return false;
        const int dp = I.prec == GPA_PREC_BF16_TC ? gmm_dp(I.d) : batched_dp(I.d), c = class_of(dp);
        BInst& B = P.inst[i];
        B.n = I.n;
        B.d = I.d;
        B.k = I.k;
        B.m = I.m;
        B.dp = dp;
        B.gamma = I.gamma;
        B.cw = gmm_prior_const(I.d, I.m, I.gamma);
        B.seed = I.seed;
        B.ntiles128 = (int)((I.n + 127) / 128);
        if (I.prec == GPA_PREC_BF16_TC) {  // prep and finalize items only; pointers bound below
            P.cat[dp == 64 ? 0 : 1].members.push_back(i);
            for (int kk = 0; kk < I.k; ++kk) P.items[c][kPhPrep].push_back({i, kk, 0, 0});
            for (int kk = 0; kk < I.k; ++kk) P.items[c][kPhFin].push_back({i, kk, 0, 0});
            P.items[c][kPhFin].push_back({i, -1, 0, 0});  // objective
            continue;
        }
        const int64_t ntiles64 = (I.n + bwd_tpb(dp) - 1) / bwd_tpb(dp);  // backward tiles
        const int64_t chunk_points = O.chunk_points[c];
        int nch = (int)((I.n + chunk_points - 1) / chunk_points);
        nch = std::max(1, std::min(nch, kGmmMaxChunks));
        nch = (int)std::min<int64_t>(nch, ntiles64);
        B.tiles_per_chunk = (ntiles64 + nch - 1) / nch;
        B.nchunks = (int)((ntiles64 + B.tiles_per_chunk - 1) / B.tiles_per_chunk);
        const bool small = O.small_groups[c] && use_small_groups(dp, I.k);
        const int gc = small ? small_gc_of(dp) : gc_of(dp);
        const int groups = (I.k + gc - 1) / gc;
        for (int kk = 0; kk < I.k; ++kk) P.items[c][kPhPrep].push_back({i, kk, 0, 0});
        for (int t = 0; t < B.ntiles128; ++t) P.items[c][kPhFwd].push_back({i, t, 0, 0});
        for (int g = 0; g < groups; ++g)
            for (int ch = 0; ch < B.nchunks; ++ch) P.items[c][small ? kPhBwdSmall : kPhBwd].push_back({i, g, ch, 0});
        for (int kk = 0; kk < I.k; ++kk) P.items[c][kPhFin].push_back({i, kk, 0, 0});
        P.items[c][kPhFin].push_back({i, -1, 0, 0});  // objective
    }
    // longest-processing-time order for the forward and backward lists
    for (int c = 0; c < kClasses; ++c) {
        auto cost_f = [&](const BItem& w) { return (double)P.inst[w.inst].k; };
        auto cost_b = [&](const BItem& w) {
            const BInst& B = P.inst[w.inst];
            const int64_t ntiles64 = (B.n + bwd_tpb(B.dp) - 1) / bwd_tpb(B.dp);
            const int64_t t0 = (int64_t)w.b * B.tiles_per_chunk;
            return (double)std::max<int64_t>(0, std::min<int64_t>(ntiles64, t0 + B.tiles_per_chunk) - t0);
        };
        std::stable_sort(P.items[c][kPhFwd].begin(), P.items[c][kPhFwd].end(),
                         [&](const BItem& u, const BItem& v) { return cost_f(u) > cost_f(v); });
        for (int ph : {kPhBwd, kPhBwdSmall})
            std::stable_sort(P.items[c][ph].begin(), P.items[c][ph].end(),
                             [&](const BItem& u, const BItem& v) { return cost_b(u) > cost_b(v); });
    }
    // tensor-core instances: a concatenated class per padded dimension where
    // its responsibilities fit, else the per-instance path
    for (int q = 0; q < 2; ++q) {
        CatPlan& C = P.cat[q];
        C.tdp = q == 0 ? 64 : 128;
        if (C.members.empty()) continue;
        int64_t np = 0, kr = 0;
        for (int i : C.members) {
            np += (in[i].n + 127) / 128 * 128;
            kr = std::max<int64_t>(kr, (in[i].k + 15) / 16 * 16);
        }
        C.on = (size_t)kr * (size_t)np * 2 <= kCatRBytes;
        if (!C.on) {
            for (int i : C.members) {
                P.tc.push_back(i);
                P.inst[i].nchunks = gmm_tc_bwd_nchunks(in[i].n, in[i].d, in[i].k);
            }
            continue;
        }
        C.np = np;
        C.kr = kr;
        const int64_t chunk_points = O.chunk_points[class_of(C.tdp)];
        int64_t xoff = 0, xtoff = 0, koff = 0;
        for (int m = 0; m < (int)C.members.size(); ++m) {
            const int i = C.members[m];
            const gpa_gmm_instance& I = in[i];
            BInst& B = P.inst[i];
            TcCatInst T{};
            T.n = I.n;
            T.d = I.d;
            T.k = I.k;
            T.xoff = xoff;
            T.xtoff = xtoff;
            T.koff = (int)koff;
            const int krr = (I.k + 15) / 16 * 16;
            T.kn = krr < 256 ? krr : 256;
            T.seed = (float)I.seed;
            const int gg = gmm_tc_cat_gram_groups(I.d, I.k);  // product groups x component groups
            const int nkg = (krr + 255) / 256;
            T.ng = gg / nkg;
            const int64_t ntiles64 = (I.n + 63) / 64;
            int nch = (int)std::min<int64_t>(std::max<int64_t>(1, (I.n + chunk_points - 1) / chunk_points),
                                             kGmmMaxChunks);
            nch = (int)std::min<int64_t>(nch, ntiles64);
            T.tpc = (ntiles64 + nch - 1) / nch;
            T.nchunks = (int)((ntiles64 + T.tpc - 1) / T.tpc);
            B.nchunks = T.nchunks;
            const int64_t npad = (I.n + 127) / 128 * 128;
            for (int64_t t = 0; t < npad / 128; ++t) C.tile_inst.push_back(m);
            for (int t = 0; t < B.ntiles128; ++t) C.fwd_tiles.push_back(make_int2(m, t));
            for (int bx = 0; bx < gg; ++bx)
                for (int ch = 0; ch < T.nchunks; ++ch) C.gram_items.push_back(make_int4(m, bx, ch, 0));
            C.cinst.push_back(T);
            xoff += npad;
            xtoff += npad * I.d;
            koff += I.k;
        }
        C.kc = koff;
        // longest first: forward tiles by rounds (components), gram items by tiles per chunk
        std::stable_sort(C.fwd_tiles.begin(), C.fwd_tiles.end(),
                         [&](int2 u, int2 v) { return C.cinst[u.x].k > C.cinst[v.x].k; });
        std::stable_sort(C.gram_items.begin(), C.gram_items.end(),
                         [&](int4 u, int4 v) { return C.cinst[u.x].tpc > C.cinst[v.x].tpc; });
    }
    for (int c = 0; c < kClasses; ++c)
        for (int ph = 0; ph < kPhases; ++ph) {
            P.off_items[c][ph] = off;
            off = a256(off + sizeof(BItem) * P.items[c][ph].size());
        }
    for (CatPlan& C : P.cat) {
        if (!C.on) continue;
        C.off_cinst = off;
        off = a256(off + sizeof(TcCatInst) * C.cinst.size());
        C.off_tile_inst = off;
        off = a256(off + sizeof(int) * C.tile_inst.size());
        C.off_fwd_tiles = off;
        off = a256(off + sizeof(int2) * C.fwd_tiles.size());
        C.off_gram_items = off;
        off = a256(off + sizeof(int4) * C.gram_items.size());
    }
    P.off_counters = off;
    off = a256(off + sizeof(int) * kClasses * kPhases);
    // Accum partials of every instance, contiguous so that one memset clears them
    P.off_partials = off;
    auto in_cat = [&](int i) {
        if (in[i].prec != GPA_PREC_BF16_TC) return false;
        return P.cat[P.inst[i].dp == 64 ? 0 : 1].on;
    };
    for (int i = 0; i < n_inst; ++i) {
        if (in[i].prec == GPA_PREC_BF16_TC && !in_cat(i)) continue;
        BInst& B = P.inst[i];
        B.bS = (float*)(base + off);
        off = a256(off + sizeof(float) * (size_t)B.nchunks * B.k * nblk(B.dp) * 64);
        B.bM = (float*)(base + off);
        off = a256(off + sizeof(float) * (size_t)B.nchunks * B.k * (B.dp + 1));
    }
    P.partial_bytes = off - P.off_partials;
    P.off_regions = off;
    for (int i = 0; i < n_inst; ++i) {
        if (in[i].prec == GPA_PREC_BF16_TC) continue;
        BInst& B = P.inst[i];
        const gpa_gmm_instance& I = in[i];
        B.x = I.x; B.alpha = I.alpha; B.mu = I.mu; B.q = I.q; B.l = I.l;
        B.d_alpha = I.d_alpha; B.d_mu = I.d_mu; B.d_q = I.d_q; B.d_l = I.d_l; B.out = I.out;
        B.rec = (float*)(base + off);  off = a256(off + sizeof(float) * (size_t)B.k * (B.dp * B.dp + B.dp + 4));
        B.scal = (double*)(base + off); off = a256(off + sizeof(double) * 8);
        B.lpk = (double*)(base + off);  off = a256(off + sizeof(double) * (size_t)B.k);
        B.fwd = (double*)(base + off);  off = a256(off + sizeof(double) * (size_t)B.ntiles128);
        B.lse = (float*)(base + off);   off = a256(off + sizeof(float) * (size_t)B.n);
        B.lj = (float*)(base + off);    off = a256(off + sizeof(float) * (size_t)B.n * B.k);
    }
    // concatenated tensor-core classes: shared buffers, per-instance scalars
    for (CatPlan& C : P.cat) {
        if (!C.on) continue;
        const int tdp = C.tdp, rec_len = tdp * tdp + tdp + 4;
        int64_t pairs = 0, xtf = 0;
        for (int i : C.members) {
            // log-joint rows padded to whole 128-point tiles (16-byte aligned rows)
            pairs += (in[i].n + 127) / 128 * 128 * (int64_t)in[i].k;
            xtf += (in[i].n + 127) / 128 * 128 * (int64_t)in[i].d;
        }
        C.off_rec = off; off = a256(off + sizeof(float) * (size_t)C.kc * rec_len);
        C.off_tails = off; off = a256(off + sizeof(float) * (size_t)C.kc * (tdp + 4));
        C.off_xb = off;  off = a256(off + 2 * (size_t)C.np * tdp);
        C.off_xl = off;  off = a256(off + 2 * (size_t)C.np * tdp);
        C.off_qb = off;  off = a256(off + 2 * (size_t)C.kc * tdp * tdp);
        C.off_ql = off;  off = a256(off + 2 * (size_t)C.kc * tdp * tdp);
        C.off_rb = off;  off = a256(off + 2 * (size_t)C.kr * C.np);
        C.off_xt = off;  off = a256(off + 2 * (size_t)xtf);  // bf16
        C.off_lse = off; off = a256(off + sizeof(float) * (size_t)C.np);
        C.off_lj = off;  off = a256(off + sizeof(float) * (size_t)pairs);
        int64_t ljo = 0;
        for (int m = 0; m < (int)C.members.size(); ++m) {
            const int i = C.members[m];
            const gpa_gmm_instance& I = in[i];
            BInst& B = P.inst[i];
            TcCatInst& T = C.cinst[m];
            B.x = I.x; B.alpha = I.alpha; B.mu = I.mu; B.q = I.q; B.l = I.l;
            B.d_alpha = I.d_alpha; B.d_mu = I.d_mu; B.d_q = I.d_q; B.d_l = I.d_l; B.out = I.out;
            B.rec = (float*)(base + C.off_rec) + (size_t)T.koff * rec_len;
            B.scal = (double*)(base + off); off = a256(off + sizeof(double) * 8);
            B.lpk = (double*)(base + off);  off = a256(off + sizeof(double) * (size_t)B.k);
            B.fwd = (double*)(base + off);  off = a256(off + sizeof(double) * (size_t)B.ntiles128);
            B.lse = (float*)(base + C.off_lse) + T.xoff;
            B.lj = (float*)(base + C.off_lj) + ljo;
            ljo += (I.n + 127) / 128 * 128 * (int64_t)I.k;
            T.x = I.x;
            T.lj = B.lj;
            T.lse = B.lse;
            T.fwd = B.fwd;
            T.bS = B.bS;
            T.bM = B.bM;
        }
    }
    // tensor-core regions: the per-call layout of each instance; the batched
    // prep and finalize read and write its records, scalars and partial sums there
    for (int i : P.tc) {
        const gpa_gmm_instance& I = in[i];
        BInst& B = P.inst[i];
        const GmmLayout L = gmm_layout(I.n, I.d, I.k, 0);
        char* r = base + off;
        P.tc_off.push_back(off);
        B.x = I.x; B.alpha = I.alpha; B.mu = I.mu; B.q = I.q; B.l = I.l;
        B.d_alpha = I.d_alpha; B.d_mu = I.d_mu; B.d_q = I.d_q; B.d_l = I.d_l; B.out = I.out;
        B.rec = (float*)(r + L.off_rec);
        B.scal = (double*)(r + L.off_scal);
        B.lpk = (double*)(r + L.off_lpk);
        B.fwd = (double*)(r + L.off_fwd);
        B.bS = (float*)(r + L.off_bS);
        B.bM = (float*)(r + L.off_bM);
        B.lse = nullptr;
        B.lj = nullptr;
        off = a256(off + tc_instance_bytes(I));
    }
    P.total = off;
    return true;
}

// Fork the lanes from s and enqueue the contractions of the tensor-core
// instances on them (their prep ran before, their finalize runs after the
// join); the caller enqueues the FP32 classes on s meanwhile and then calls
// tc_join.
int tc_fork_and_run(const gpa_gmm_instance* in, const Plan& P, char* ws, int32_t* status, cudaStream_t s) {
    if (P.tc.empty()) return GPA_OK;
    TcLanes* T = tc_lanes(false);
    if (!T) return GPA_ERR_CUDA;  // gmm_batched_prepare makes the lanes
    const int lanes = std::min<int>(kTcLanes, (int)P.tc.size());
    if (cudaEventRecord(T->fork, s) != cudaSuccess) return GPA_ERR_CUDA;
    for (int j = 0; j < lanes; ++j)
        if (cudaStreamWaitEvent(T->st[j], T->fork, 0) != cudaSuccess) return GPA_ERR_CUDA;
    // longest instances first, dealt round-robin over the lanes
    std::vector<int> order(P.tc.size());
    for (size_t t = 0; t < order.size(); ++t) order[t] = (int)t;
    std::stable_sort(order.begin(), order.end(), [&](int u, int v) {
        return in[P.tc[u]].n * in[P.tc[u]].k > in[P.tc[v]].n * in[P.tc[v]].k;
    });
    int rc = GPA_OK;
    for (size_t t = 0; t < order.size() && rc == GPA_OK; ++t) {
        const int j = (int)(t % lanes);
        const gpa_gmm_instance& I = in[P.tc[order[t]]];
        GmmArgs A{};
        A.x = I.x; A.alpha = I.alpha; A.mu = I.mu; A.q = I.q; A.l = I.l; A.n = I.n; A.d = I.d; A.k = I.k;
        A.gamma = I.gamma; A.m = I.m; A.seed = I.seed; A.out = I.out; A.status = status;
        A.d_alpha = I.d_alpha; A.d_mu = I.d_mu; A.d_q = I.d_q; A.d_l = I.d_l;
        const GmmLayout L = gmm_layout(I.n, I.d, I.k, 0);
        rc = gmm_tc_vjp_run(A, L, ws + P.tc_off[order[t]], tc_instance_bytes(I), T->st[j], kGmmStageCore);
    }
    return rc;
}

// Join every forked lane back into s (also after an error, so that no lane
// stays forked, which would leave a graph capture unjoined).
int tc_join(const Plan& P, cudaStream_t s) {
    if (P.tc.empty()) return GPA_OK;
    TcLanes* T = tc_lanes(false);
    if (!T) return GPA_ERR_CUDA;
    const int lanes = std::min<int>(kTcLanes, (int)P.tc.size());
    for (int j = 0; j < lanes; ++j)
        if (cudaEventRecord(T->join[j], T->st[j]) != cudaSuccess || cudaStreamWaitEvent(s, T->join[j], 0) != cudaSuccess)
            return GPA_ERR_CUDA;
    return GPA_OK;
}

// ---- persistent kernels -----------------------------------------------------------
__device__ __forceinline__ int next_item(int* counter) {
    __shared__ int s_item;
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    return it;
}

template <int DP>
__global__ void __launch_bounds__(128) batched_prep_kernel(const BInst* __restrict__ inst,
                                                           const BItem* __restrict__ items, int n_items,
                                                           int* counter) {
    for (;;) {
        const int it = next_item(counter);
        if (it >= n_items) break;
        const BItem w = items[it];
        const BInst& B = inst[w.inst];
        gmm_prep_kernel_body<DP>(B.alpha, B.mu, B.q, B.l, B.d, B.k, B.gamma, B.m, B.cw, B.rec, B.lpk, B.scal,
                                 (unsigned)w.a);
        __syncthreads();
    }
}

template <int DP>
__global__ void __launch_bounds__(256, (DP <= 64 ? 2 : 1))
    batched_fwd_kernel(const BInst* __restrict__ inst, const BItem* __restrict__ items, int n_items, int* counter,
                       int32_t* status) {
    for (;;) {
        const int it = next_item(counter);
        if (it >= n_items) break;
        const BItem w = items[it];
        const BInst& B = inst[w.inst];
        gmm_fwd_kernel_body<DP>(B.x, B.n, B.d, B.k, B.rec, B.lj, B.n, B.lse, B.fwd, 0, status, (unsigned)w.a);
        __syncthreads();
    }
}

template <int DP, int GCX = 0>
__global__ void __launch_bounds__(Bwd<DP, GCX>::THREADS, Bwd<DP, GCX>::MINB)
    batched_bwd_kernel(const BInst* __restrict__ inst, const BItem* __restrict__ items, int n_items,
                       int* counter) {
    for (;;) {
        const int it = next_item(counter);
        if (it >= n_items) break;
        const BItem w = items[it];
        const BInst& B = inst[w.inst];
        gmm_bwd_kernel_body<DP, Bwd<DP>::UNROLL_BATCHED, GCX>(B.x, B.n, B.d, B.k, B.lj, B.n, B.lse, (float)B.seed,
                                                            B.tiles_per_chunk, B.bS, B.bM, (unsigned)w.a,
                                                            (unsigned)w.b);
        __syncthreads();
    }
}

template <int DP>
__global__ void __launch_bounds__(256) batched_fin_kernel(const BInst* __restrict__ inst,
                                                          const BItem* __restrict__ items, int n_items,
                                                          int* counter) {
    for (;;) {
        const int it = next_item(counter);
        if (it >= n_items) break;
        const BItem w = items[it];
        const BInst& B = inst[w.inst];
        if (w.a < 0) {
            if (B.out) gmm_objective_finalize_kernel_body(B.fwd, B.ntiles128, B.lpk, B.k, B.scal, B.n, B.d, B.out, 0u);
        } else {
            gmm_finalize_kernel_body<DP>(B.alpha, B.mu, B.q, B.l, B.d, B.k, B.n, B.gamma, B.m, B.seed, B.bS, B.bM,
                                         B.nchunks, B.scal, B.d_alpha, B.d_mu, B.d_q, B.d_l, 0, nullptr,
                                         (unsigned)w.a);
        }
        __syncthreads();
    }
}

// ---- D <= 8 ------------------------------------------------------------------------
// Forward: one thread per point, the point's 8 coordinates in registers, the
// component records (Q^T, b, constant) staged kD8Stage at a time in shared
// memory and read as broadcasts. z = Q x - b in packed pairs of rows over the
// lower triangle (column c touches rows c.. only), then the log-joint and the
// online logsumexp as in the other forward kernels.
__global__ void __launch_bounds__(128) batched_fwd8_kernel(const BInst* __restrict__ inst,
                                                           const BItem* __restrict__ items, int n_items,
                                                           int* counter) {
    __shared__ __align__(16) float qs[kD8Stage * kD8Rec];
    __shared__ double wsum[4];
    for (;;) {
        const int it = next_item(counter);
        if (it >= n_items) break;
        const BItem w = items[it];
        const BInst& B = inst[w.inst];
        const int64_t p = (int64_t)w.a * kD8Points + threadIdx.x;
        const bool valid = p < B.n;
        float xv[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) xv[c] = (valid && c < B.d) ? __ldg(B.x + p * B.d + c) : 0.f;
        Lse st;
        st.init();
        for (int c0 = 0; c0 < B.k; c0 += kD8Stage) {
            const int nc = min(kD8Stage, B.k - c0);
            __syncthreads();  // the previous stage's readers are done
            const float4* src = reinterpret_cast<const float4*>(B.rec + (size_t)c0 * kD8Rec);
            for (int e = threadIdx.x; e < nc * (kD8Rec / 4); e += 128)
                reinterpret_cast<float4*>(qs)[e] = __ldg(src + e);
            __syncthreads();
            for (int j = 0; j < nc; ++j) {
                const float* R = qs + j * kD8Rec;  // Qt[c][r] at 8 c + r, b at 64, constant at 72
                const float4 b0 = *reinterpret_cast<const float4*>(R + 64);
                const float4 b1 = *reinterpret_cast<const float4*>(R + 68);
                float2 z[4] = {make_float2(-b0.x, -b0.y), make_float2(-b0.z, -b0.w), make_float2(-b1.x, -b1.y),
                               make_float2(-b1.z, -b1.w)};
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float4 q0 = *reinterpret_cast<const float4*>(R + 8 * c);
                    const float4 q1 = *reinterpret_cast<const float4*>(R + 8 * c + 4);
                    const float2 qp[4] = {make_float2(q0.x, q0.y), make_float2(q0.z, q0.w), make_float2(q1.x, q1.y),
                                          make_float2(q1.z, q1.w)};
                    const float2 x2 = make_float2(xv[c], xv[c]);
#pragma unroll
                    for (int i = c / 2; i < 4; ++i) z[i] = __ffma2_rn(x2, qp[i], z[i]);
                }
                float2 s2 = __fmul2_rn(z[0], z[0]);
#pragma unroll
                for (int i = 1; i < 4; ++i) s2 = __ffma2_rn(z[i], z[i], s2);
                const float v = R[72] - 0.5f * (s2.x + s2.y);
                if (valid) {
                    if (B.lj) B.lj[(int64_t)(c0 + j) * B.n + p] = v;
                    st.add(v);
                }
            }
        }
        double v = 0.0;
        if (valid) {
            const float lv = st.value();
            if (B.lse) B.lse[p] = lv;
            v = (double)lv;
        }
        v = warp_sum(v);
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) B.fwd[w.a] = wsum[0] + wsum[1] + wsum[2] + wsum[3];
    }
}

// Backward Accum: item (instance, group of up to kD8Group components, point
// chunk). The nc components of the group share the CTA's 128 threads: thread
// t takes component t % nc and every ps-th point of each tile from t / nc
// (ps = 128 / nc slices), so a group of few components still keeps most
// threads busy. Per point and component: r = seed exp(s - lse), y = r x,
// S += y x^T (lower triangle, 36 sums), m += y, R += r. The slices' sums are
// then combined in slice order and added into the chunk's partial sums.
constexpr int kD8Sums = 36 + 8 + 1;
__global__ void __launch_bounds__(128) batched_bwd8_kernel(const BInst* __restrict__ inst,
                                                           const BItem* __restrict__ items, int n_items,
                                                           int* counter) {
    __shared__ __align__(16) float xs[kD8Points * 8];
    __shared__ float rs[kD8Points * kD8Group];
    __shared__ float lse_s[kD8Points];
    __shared__ float red[128 * kD8Sums];
    const int tid = threadIdx.x;
    for (;;) {
        const int it = next_item(counter);
        if (it >= n_items) break;
        const BItem w = items[it];
        const BInst& B = inst[w.inst];
        const int kg0 = w.a * kD8Group, nc = min(kD8Group, B.k - kg0), ps = 128 / nc;
        const int c = tid % nc, sl = tid / nc;
        const bool active = sl < ps;
        const int64_t ntiles = (B.n + kD8Points - 1) / kD8Points;
        const int64_t t0 = (int64_t)w.b * B.tiles_per_chunk, t1 = min64(ntiles, t0 + B.tiles_per_chunk);
        const float seed = (float)B.seed;
        float S[36], m[8], R = 0.f;
#pragma unroll
        for (int e = 0; e < 36; ++e) S[e] = 0.f;
#pragma unroll
        for (int e = 0; e < 8; ++e) m[e] = 0.f;
        for (int64_t t = t0; t < t1; ++t) {
            const int64_t p0 = t * kD8Points;
            __syncthreads();  // the previous tile's readers are done
            for (int e = tid; e < kD8Points * 8; e += 128) {
                const int pp = e >> 3, cc = e & 7;
                xs[e] = (p0 + pp < B.n && cc < B.d) ? __ldg(B.x + (p0 + pp) * B.d + cc) : 0.f;
            }
            lse_s[tid] = p0 + tid < B.n ? __ldg(B.lse + p0 + tid) : 0.f;
            __syncthreads();
            for (int e = tid; e < nc * kD8Points; e += 128) {
                const int cc = e / kD8Points, pp = e % kD8Points;
                float r = 0.f;
                if (p0 + pp < B.n) r = seed * expf(__ldg(B.lj + (int64_t)(kg0 + cc) * B.n + p0 + pp) - lse_s[pp]);
                rs[pp * kD8Group + cc] = r;
            }
            __syncthreads();
            if (active)
                for (int pp = sl; pp < kD8Points; pp += ps) {
                    const float r = rs[pp * kD8Group + c];
                    const float4 xa = *reinterpret_cast<const float4*>(xs + pp * 8);
                    const float4 xb = *reinterpret_cast<const float4*>(xs + pp * 8 + 4);
                    const float x[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
                    R += r;
#pragma unroll
                    for (int a = 0; a < 8; ++a) {
                        const float y = r * x[a];
                        m[a] += y;
#pragma unroll
                        for (int b = 0; b <= a; ++b) S[a * (a + 1) / 2 + b] = fmaf(y, x[b], S[a * (a + 1) / 2 + b]);
                    }
                }
        }
        __syncthreads();
        if (active) {
            float* o = red + (sl * nc + c) * kD8Sums;
#pragma unroll
            for (int e = 0; e < 36; ++e) o[e] = S[e];
#pragma unroll
            for (int e = 0; e < 8; ++e) o[36 + e] = m[e];
            o[44] = R;
        }
        __syncthreads();
        for (int e2 = tid; e2 < nc * kD8Sums; e2 += 128) {
            const int cc = e2 / kD8Sums, e = e2 % kD8Sums;
            float v = 0.f;
            for (int s2 = 0; s2 < ps; ++s2) v += red[(s2 * nc + cc) * kD8Sums + e];
            const int64_t base = (int64_t)w.b * B.k + kg0 + cc;
            if (e < 36) {
                int a = 0, b = e;
                while (b > a) {
                    ++a;
                    b -= a;
                }
                B.bS[base * 64 + a * 8 + b] += v;
            } else {
                B.bM[base * 9 + (e - 36)] += v;  // m at 0..7, R at 8
            }
        }
    }
}

// ---- host -------------------------------------------------------------------------
template <typename K>
bool smem_attr(K kern, size_t bytes) {
    if (bytes <= 48 * 1024) return true;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
}

int sms() {
    int dev = 0, n = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

template <typename K>
unsigned persistent_grid(K kern, int threads, size_t smem, int n_items, int ctas_per_sm) {
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    occ = std::max(1, occ);
    if (ctas_per_sm > 0) occ = std::min(occ, ctas_per_sm);
    return (unsigned)std::max(1, std::min(n_items, sms() * occ));
}

// The phases of one class: prep and finalize also cover the class's
// tensor-core instances, forward and backward only its FP32 ones.
template <int DP>
struct ClassRun {
    const Plan& P;
    char* ws;
    int c;
    const BInst* inst() const { return (const BInst*)(ws + P.off_desc); }
    int* counter(int ph) const { return (int*)(ws + P.off_counters) + c * kPhases + ph; }
    const BItem* items(int ph) const { return (const BItem*)(ws + P.off_items[c][ph]); }
    int count(int ph) const { return (int)P.items[c][ph].size(); }

    int prep(cudaStream_t s) const {
        if (count(kPhPrep) == 0) return GPA_OK;
        auto k = batched_prep_kernel<DP>;
        const unsigned g = persistent_grid(k, 128, 0, count(kPhPrep), 0);
        GPA_LAUNCH("gmm_batched_prep", s,
                   k<<<g, 128, 0, s>>>(inst(), items(kPhPrep), count(kPhPrep), counter(kPhPrep)));
        return GPA_OK;
    }
    template <int GCX>
    int bwd(int ph, int ctas_per_sm, cudaStream_t s) const {
        if (count(ph) == 0) return GPA_OK;
        using C = Bwd<DP, GCX>;
        auto kb = batched_bwd_kernel<DP, GCX>;
        if (!smem_attr(kb, C::SMEM)) return GPA_ERR_CUDA;
        const unsigned gb = persistent_grid(kb, C::THREADS, C::SMEM, count(ph), ctas_per_sm);
        GPA_LAUNCH("gmm_batched_bwd", s, kb<<<gb, C::THREADS, C::SMEM, s>>>(inst(), items(ph), count(ph), counter(ph)));
        return GPA_OK;
    }
    int core(int ctas_per_sm, int32_t* status, cudaStream_t s) const {
        if (count(kPhFwd) == 0) return GPA_OK;
        if constexpr (DP == 8) {
            (void)status;
            auto kf = batched_fwd8_kernel;
            const unsigned gf = persistent_grid(kf, 128, 0, count(kPhFwd), ctas_per_sm);
            GPA_LAUNCH("gmm_batched_fwd", s,
                       kf<<<gf, 128, 0, s>>>(inst(), items(kPhFwd), count(kPhFwd), counter(kPhFwd)));
            auto kb = batched_bwd8_kernel;
            const unsigned gb = persistent_grid(kb, 128, 0, count(kPhBwd), ctas_per_sm);
            GPA_LAUNCH("gmm_batched_bwd", s,
                       kb<<<gb, 128, 0, s>>>(inst(), items(kPhBwd), count(kPhBwd), counter(kPhBwd)));
            return GPA_OK;
        } else {
            auto kf = batched_fwd_kernel<DP>;
            if (!smem_attr(kf, Fwd<DP>::SMEM)) return GPA_ERR_CUDA;
            const unsigned gf = persistent_grid(kf, Fwd<DP>::THREADS, Fwd<DP>::SMEM, count(kPhFwd), ctas_per_sm);
            GPA_LAUNCH("gmm_batched_fwd", s,
                       kf<<<gf, Fwd<DP>::THREADS, Fwd<DP>::SMEM, s>>>(inst(), items(kPhFwd), count(kPhFwd),
                                                                      counter(kPhFwd), status));
            int rc = bwd<0>(kPhBwd, ctas_per_sm, s);
            if (rc) return rc;
            if constexpr (DP == 16) return bwd<kSmallGc16>(kPhBwdSmall, ctas_per_sm, s);
            if constexpr (DP == 32) return bwd<kSmallGc32>(kPhBwdSmall, ctas_per_sm, s);
            return GPA_OK;
        }
    }
    int fin(cudaStream_t s) const {
        if (count(kPhFin) == 0) return GPA_OK;
        const size_t smem = gmm_finalize_smem<DP>();
        auto k = batched_fin_kernel<DP>;
        if (!smem_attr(k, smem)) return GPA_ERR_CUDA;
        const unsigned g = persistent_grid(k, 256, smem, count(kPhFin), 0);
        GPA_LAUNCH("gmm_batched_finalize", s,
                   k<<<g, 256, smem, s>>>(inst(), items(kPhFin), count(kPhFin), counter(kPhFin)));
        return GPA_OK;
    }
};

int check_instances(const gpa_gmm_instance* in, int n_inst) {
    if (!in || n_inst < 1 || n_inst > (1 << 20)) return GPA_ERR_ARG;
    for (int i = 0; i < n_inst; ++i) {
        const gpa_gmm_instance& I = in[i];
        if (!I.x || !I.alpha || !I.mu || !I.q || (I.d > 1 && !I.l) || !I.d_alpha || !I.d_mu || !I.d_q ||
            (I.d > 1 && !I.d_l))
            return GPA_ERR_ARG;
        if (I.n < 1 || I.n > INT32_MAX || I.d < 1 || I.d > 128 || I.k < 1 || I.k > 4096 || !(I.gamma > 0.0))
            return GPA_ERR_ARG;
        if (I.prec != GPA_PREC_FP32 && I.prec != GPA_PREC_BF16_TC) return GPA_ERR_ARG;
        if (I.prec == GPA_PREC_BF16_TC && !gmm_tc_supported(I.d)) return GPA_ERR_UNSUPPORTED;
    }
    return GPA_OK;
}

}  // namespace
}  // namespace gpa

using namespace gpa;

namespace {
gpa_batched_opts uniform_opts(int64_t chunk_points, int32_t ctas_per_sm) {
    gpa_batched_opts O;
    for (int c = 0; c < kClasses; ++c) {
        O.chunk_points[c] = chunk_points;
        O.ctas_per_sm[c] = ctas_per_sm;
        O.small_groups[c] = 0;
    }
    return O;
}
bool opts_ok(const gpa_batched_opts* O) {
    if (!O) return false;
    for (int c = 0; c < kClasses; ++c)
        if (O->chunk_points[c] < 64 || O->ctas_per_sm[c] < 0) return false;
    return true;
}
}  // namespace

extern "C" size_t gpa_gmm_batched_workspace_bytes_opts(const gpa_gmm_instance* inst, int32_t n_inst,
                                                       const gpa_batched_opts* opts) {
    if (check_instances(inst, n_inst) || !opts_ok(opts)) return 0;
    Plan P;
    if (!make_plan(inst, n_inst, *opts, nullptr, P)) return 0;
    return P.total + 256;
}

extern "C" int gmm_batched_prepare_opts(const gpa_gmm_instance* inst, int32_t n_inst, const gpa_batched_opts* opts,
                                        void* ws, size_t ws_bytes, gpa_stream_t stream) {
    int rc = check_instances(inst, n_inst);
    if (rc) return rc;
    if (!ws || !opts_ok(opts)) return GPA_ERR_ARG;
    if (((uintptr_t)ws) & 255) return GPA_ERR_ALIGN;
    Plan P;
    if (!make_plan(inst, n_inst, *opts, (char*)ws, P)) return GPA_ERR_ARG;
    if (ws_bytes < P.total) return GPA_ERR_WORKSPACE;
    if (!P.tc.empty() && !tc_lanes(true)) return GPA_ERR_CUDA;
    // host image of descriptors and work lists, copied in one transfer
    std::vector<char> img(P.off_regions, 0);
    memcpy(img.data() + P.off_desc, P.inst.data(), sizeof(BInst) * P.inst.size());
    for (int c = 0; c < kClasses; ++c)
        for (int ph = 0; ph < kPhases; ++ph)
            if (!P.items[c][ph].empty())
                memcpy(img.data() + P.off_items[c][ph], P.items[c][ph].data(),
                       sizeof(BItem) * P.items[c][ph].size());
    for (const CatPlan& C : P.cat) {
        if (!C.on) continue;
        memcpy(img.data() + C.off_cinst, C.cinst.data(), sizeof(TcCatInst) * C.cinst.size());
        memcpy(img.data() + C.off_tile_inst, C.tile_inst.data(), sizeof(int) * C.tile_inst.size());
        memcpy(img.data() + C.off_fwd_tiles, C.fwd_tiles.data(), sizeof(int2) * C.fwd_tiles.size());
        memcpy(img.data() + C.off_gram_items, C.gram_items.data(), sizeof(int4) * C.gram_items.size());
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(ws, img.data(), P.off_partials, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        (void)cudaGetLastError();
        return GPA_ERR_CUDA;
    }
    return GPA_OK;
}

extern "C" int gmm_batched_vjp_opts(const gpa_gmm_instance* inst, int32_t n_inst, const gpa_batched_opts* opts,
                                    void* ws, size_t ws_bytes, int32_t* dev_status, gpa_stream_t stream) {
    int rc = check_instances(inst, n_inst);
    if (rc) return rc;
    if (!ws || !opts_ok(opts)) return GPA_ERR_ARG;
    if (((uintptr_t)ws) & 255) return GPA_ERR_ALIGN;
    Plan P;
    if (!make_plan(inst, n_inst, *opts, (char*)ws, P)) return GPA_ERR_ARG;
    if (ws_bytes < P.total) return GPA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync((char*)ws + P.off_counters, 0, sizeof(int) * kClasses * kPhases, s) != cudaSuccess ||
        cudaMemsetAsync((char*)ws + P.off_partials, 0, P.partial_bytes, s) != cudaSuccess)
        return GPA_ERR_CUDA;
    char* w = (char*)ws;
    const int* cps = opts->ctas_per_sm;
    const ClassRun<8> c8{P, w, 0};
    const ClassRun<16> c16{P, w, 1};
    const ClassRun<32> c32{P, w, 2};
    const ClassRun<64> c64{P, w, 3};
    const ClassRun<128> c128{P, w, 4};
    // parameter expansion of every instance, then the tensor-core contractions
    // on the forked lanes concurrently with the FP32 classes on s, then every
    // instance's finalize
    if ((rc = c8.prep(s)) || (rc = c16.prep(s)) || (rc = c32.prep(s)) || (rc = c64.prep(s)) || (rc = c128.prep(s)))
        return rc;
    rc = tc_fork_and_run(inst, P, w, dev_status, s);
    for (const CatPlan& C : P.cat) {  // concatenated tensor-core classes, one launch per stage
        if (rc || !C.on) continue;
        TcCatClass T{};
        T.tdp = C.tdp;
        T.np = C.np;
        T.kc = C.kc;
        T.kr = C.kr;
        T.inst = (const TcCatInst*)(w + C.off_cinst);
        T.tile_inst = (const int*)(w + C.off_tile_inst);
        T.fwd_tiles = (const int2*)(w + C.off_fwd_tiles);
        T.gram_items = (const int4*)(w + C.off_gram_items);
        T.n_fwd = (int)C.fwd_tiles.size();
        T.n_gram = (int)C.gram_items.size();
        T.rec = (const float*)(w + C.off_rec);
        T.tails = (float*)(w + C.off_tails);
        T.xb = w + C.off_xb;
        T.xl = w + C.off_xl;
        T.qb = w + C.off_qb;
        T.ql = w + C.off_ql;
        T.rb = w + C.off_rb;
        T.xt = w + C.off_xt;
        T.status = dev_status;
        rc = gmm_tc_cat_run(T, s);
    }
    if (!rc) rc = c8.core(cps[0], dev_status, s);
    if (!rc) rc = c16.core(cps[1], dev_status, s);
    if (!rc) rc = c32.core(cps[2], dev_status, s);
    if (!rc) rc = c64.core(cps[3], dev_status, s);
    if (!rc) rc = c128.core(cps[4], dev_status, s);
    const int jr = tc_join(P, s);
    if (rc || jr) return rc ? rc : jr;
    if ((rc = c8.fin(s)) || (rc = c16.fin(s)) || (rc = c32.fin(s)) || (rc = c64.fin(s)) || (rc = c128.fin(s)))
        return rc;
    return GPA_OK;
}

extern "C" size_t gpa_gmm_batched_workspace_bytes(const gpa_gmm_instance* inst, int32_t n_inst,
                                                  int64_t chunk_points) {
    const gpa_batched_opts O = uniform_opts(chunk_points, 0);
    return gpa_gmm_batched_workspace_bytes_opts(inst, n_inst, &O);
}

extern "C" int gmm_batched_prepare(const gpa_gmm_instance* inst, int32_t n_inst, int64_t chunk_points, void* ws,
                                   size_t ws_bytes, gpa_stream_t stream) {
    const gpa_batched_opts O = uniform_opts(chunk_points, 0);
    return gmm_batched_prepare_opts(inst, n_inst, &O, ws, ws_bytes, stream);
}

extern "C" int gmm_batched_vjp(const gpa_gmm_instance* inst, int32_t n_inst, int64_t chunk_points,
                               int32_t ctas_per_sm, void* ws, size_t ws_bytes, int32_t* dev_status,
                               gpa_stream_t stream) {
    if (ctas_per_sm < 0) return GPA_ERR_ARG;
    const gpa_batched_opts O = uniform_opts(chunk_points, ctas_per_sm);
    return gmm_batched_vjp_opts(inst, n_inst, &O, ws, ws_bytes, dev_status, stream);
}
