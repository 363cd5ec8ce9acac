// a4 + a5: TLR Cholesky factorisation, forward solve and log-determinant.
//
// Left-looking tile Cholesky (the tile DAG of Sec. 2 executed column by
// column on one GPU).  For column j, with L_ik = U_ik V_ik' for k < j:
//   T_ij = A_ij - sum_{k<j} L_ik L_jk'          (i >= j)
//        = A_ij - P_ij Q_j',  Q_j = [U_j0 | ... | U_j,j-1],
//                             P_ij = [U_i0 (V_i0' V_j0) | ... ].
// The update of the whole column panel is ONE batched GEMM (all i share Q_j);
// in the likelihood path A_ij is never stored: the GEMM epilogue evaluates
// the Matern covariance of the two locations (Eq. 4.2) and subtracts the
// product, so generation and Schur update are fused.  Then
//   L_jj = chol(T_jj)                  (dense FP64),
//   T_ij ~ U V' at accuracy tau        (recompression of the updated tile),
//   V <- L_jj^-1 V                     (so that L_ij = T_ij L_jj^-T = U V').
// Each updated tile is compressed once, after all its updates (HiCMA-style
// codes recompress after every single low-rank update instead).
#include <algorithm>
#include <cmath>
#include <exception>
#include <memory>

#include "common.cuh"
#include "compress.cuh"
#include "dense.cuh"
#include "gemm.cuh"
#include "matern.cuh"
#include "tcgemm.cuh"
#include "tlr_internal.cuh"

namespace tlr {


// blockIdx.y: descriptor; blockIdx.x strides over its columns, threads over rows.
__global__ void k_copy_batched(const CopyDesc *__restrict__ d) {
    const CopyDesc c = d[blockIdx.y];
    for (int col = blockIdx.x; col < c.n; col += gridDim.x) {
        const double *src = c.src ? c.src + (int64_t)col * c.lds : nullptr;
        double *dst = c.dst + (int64_t)col * c.ldd;
        for (int r = threadIdx.x; r < c.m; r += blockDim.x) dst[r] = src ? src[r] : 0.0;
    }
}

__global__ void k_set_identity(double *__restrict__ X, int ld, int m) {
    int c = blockIdx.x;
    for (int r = threadIdx.x; r < ld; r += blockDim.x) X[(int64_t)c * ld + r] = (r == c && c < m) ? 1.0 : 0.0;
}

void set_identity(cudaStream_t s, double *X, int ld, int m) {
    launch(k_set_identity, ld, 128, 0, s, X, ld, m);
    TLR_CHECK_LAUNCH();
}

void copy_batched(tlr_ctx *ctx, cudaStream_t s, const std::vector<CopyDesc> &descs) {
    std::vector<CopyDesc> act;
    for (const CopyDesc &c : descs)
        if (c.m > 0 && c.n > 0) act.push_back(c);
    if (act.empty()) return;
    int most = 0;
    for (const CopyDesc &c : act) most = std::max(most, c.n);
    auto *dd = (const CopyDesc *)stage_push(ctx, act.data(), act.size() * sizeof(CopyDesc), s);
    launch(k_copy_batched, dim3((unsigned)std::min(most, 128), (unsigned)act.size()), 256, 0, s, dd);
    TLR_CHECK_LAUNCH();
}

static inline double *Uslot(tlr_mat *M, int i, int j) { return M->U + slot_col(M, i, j) * M->nb; }
static inline double *Vslot(tlr_mat *M, int i, int j) { return M->V + slot_col(M, i, j) * M->nb; }
static inline const double *Uslot(const tlr_mat *M, int i, int j) { return M->U + slot_col(M, i, j) * M->nb; }
static inline const double *Vslot(const tlr_mat *M, int i, int j) { return M->V + slot_col(M, i, j) * M->nb; }

// Compact layout: every factorisation starts from the base slots with an
// empty arena; a tile whose rank exceeds its slot moves into the arena.
static void reset_slots(tlr_mat *M) {
    M->cap_overflow = false;
    if (M->base_off.empty()) return;
    M->off = M->base_off;
    M->cur_cap = M->cap;
    M->arena_next = 0;
}

static GrowSlot arena_grow(tlr_mat *M) {
    if (M->base_off.empty()) return nullptr;
    return [M](const CompressJob &J, int r, double **U, double **V) -> bool {
        const int nt = M->nt, i = (int)(J.tile_id / nt), j = (int)(J.tile_id % nt);
        const int64_t need = (r + 7) & ~7;
        if (M->arena_next + need > M->arena_cols) {
            M->cap_overflow = true;
            return false;
        }
        const int64_t k = off_index(i, j);
        M->off[(size_t)k] = M->arena_off + M->arena_next;
        M->cur_cap[(size_t)k] = (int32_t)need;
        M->arena_next += need;
        *U = Uslot(M, i, j);
        *V = Vslot(M, i, j);
        return true;
    };
}

void upload_ranks(tlr_mat *M, cudaStream_t s) {
    TLR_CUDA_TRY(cudaStreamSynchronize(s));
    TLR_CUDA_TRY(cudaMemcpy(M->ranks, M->h_ranks.data(), M->h_ranks.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice));
}

// Per-factorisation state of a group (see factor_group).
struct GroupItem {
    FactorItem *in = nullptr;
    int idx = 0;  // position in the caller's list (status word, Matern item)
    tlr_mat *M = nullptr;
    int nt = 0, nb = 0;
    int64_t n = 0;
    std::vector<int32_t> prev;  // previous ranks (input ranks for FactorMode::Tlr)
    bool have_prev = false, ahead = false, solve = false, active = true;
    GrowSlot grow;
    DevBuf panel_buf[2], panel2, xinv, ytmp, vtmp;
    float2 *Tp2 = nullptr;
    double *Xinv = nullptr;
    // per finished column k: the Gram matrix G_k = V_k' V_k of its packed V
    // factors V_k = [V_ik]_{i>k} (order of i, zero-rank tiles left out), the
    // column offset of each tile in V_k, and V_k' y_k for the fused solve
    std::vector<DevBuf> gram, vty;
    std::vector<int> gram_n;
    std::vector<std::vector<int>> gram_off;
    int r_of(int i, int k) const { return (int)M->h_ranks[(size_t)i * nt + k]; }
};

void factor_group(tlr_ctx *ctx, cudaStream_t st, std::vector<FactorItem> &list, FactorMode mode, bool df,
                  bool tc) {
    if (list.empty()) return;
    if ((int)list.size() > kMaxGroup) throw make_error(TLR_ERR_ARG, "more than %d factorisations in one call", kMaxGroup);
    if (df && mode != FactorMode::Matern) throw make_error(TLR_ERR_ARG, "paired-FP32 products need the Matern mode");
    if (tc && !df) throw make_error(TLR_ERR_ARG, "tensor-core products belong to the mixed path");
    if (mode == FactorMode::Tlr && list.size() != 1) throw make_error(TLR_ERR_ARG, "one compressed input per call");
    // tc: the panel update (the large product, on the look-ahead stream) runs
    // on the tensor cores (tcgemm.cuh) from the FP64 operands.  The small
    // products on the critical path (correction, sampling, projection,
    // V <- L^-1 V, Gram) can run there too (tcc), but measured slower at
    // n = 40,000 than paired FP32: their 128 x 32 tiles keep the tensor pipe
    // below a third of its rate and the operand splits add a launch each on
    // the critical path; they stay paired FP32.
    // The Gram matrices V_j' V_j (inner dimension the tile size, S x S
    // outputs) are the one critical-path product measured faster there
    // (13.6 -> 5.9 ms per evaluation at n = 40,000; all of them on the
    // tensor cores: 469 -> 638 ms).
    const bool tcp = tc, tcc = false, tcg = tc;
    const bool dfp = df && !tcc;  // paired-FP32 copies for the critical-path products
    const int G = (int)list.size();
    FactorStats *pstats = list[0].stats;  // profiling totals of the call
    int prof_used = 0;
    for (double &v : ctx->comp_ms) v = 0.0;
    compress_profile_reset(ctx);
    for (long long &v : ctx->comp_stats) v = 0;
    ctx->k16_ms = ctx->k16_flops = 0.0;
    ctx->k16_launches = ctx->k16_clusters = 0;
    // Look-ahead (likelihood path): the update of column j+1 by the columns
    // k < j runs on a third stream while column j is compressed (which keeps
    // most SMs idle); only the update by column j itself stays on the
    // critical path.  Two panel buffers alternate between the columns.
    // The look-ahead panel GEMM runs at the lowest stream priority with at most
    // one of its CTAs per SM, so that every SM keeps room (threads and shared
    // memory) for the compression (on a high-priority stream) and the
    // diagonal POTRF.  Two per SM left too little shared memory for the
    // compression's cluster kernels; a fixed subset of whole SMs starved the
    // compression's wide launches.
    const int ahead_ctas = ctx->ahead_ctas_per_sm;
    std::vector<std::unique_ptr<GroupItem>> items;
    int nt_max = 0;
    for (int g = 0; g < G; ++g) {
        FactorItem &F = list[(size_t)g];
        auto it = std::make_unique<GroupItem>();
        GroupItem &I = *it;
        I.in = &F;
        I.idx = g;
        I.M = F.M;
        tlr_mat *M = F.M;
        I.nt = M->nt;
        I.nb = M->nb;
        I.n = M->n;
        F.err = TLR_OK;
        F.msg.clear();
        *F.info = -1;
        // the likelihood path regenerates every tile: start from the base slots
        // (the unfused path keeps where its compressed input tiles live)
        if (mode == FactorMode::Matern) reset_slots(M);
        M->cap_overflow = false;
        I.grow = arena_grow(M);
        std::vector<int32_t> &R = M->h_ranks;  // r_ij of the factor, filled column by column
        I.prev = R;
        I.have_prev = !I.prev.empty() && I.prev.size() == (size_t)I.nt * I.nt;
        if (mode == FactorMode::Tlr && !I.have_prev) throw make_error(TLR_ERR_ARG, "matrix holds no compressed input");
        R.assign((size_t)I.nt * I.nt, 0);
        for (int t = 0; t < I.nt; ++t) R[(size_t)t * I.nt + t] = tile_rows(I.n, I.nb, t);
        I.ahead = (mode == FactorMode::Matern) && I.nt > 1;
        const size_t pb = (size_t)I.nt * I.nb * I.nb * sizeof(double);
        I.panel_buf[0].alloc(pb, st);
        if (I.ahead) I.panel_buf[1].alloc(pb, st);
        // paired-FP32 copy of the panel (mixed precision): operand of the compression products
        I.panel2.alloc(dfp ? (size_t)I.nt * I.nb * I.nb * sizeof(float2) : 0, st);
        I.Tp2 = I.panel2.as<float2>();
        I.xinv.alloc((size_t)I.nb * I.nb * sizeof(double), st);
        I.Xinv = I.xinv.as<double>();
        // fused forward solve (a5): y = L^-1 z column by column
        I.solve = (F.z != nullptr && F.y != nullptr && F.acc != nullptr);
        I.ytmp.alloc(I.solve ? (size_t)I.nb * sizeof(double) : 0, st);
        if (I.solve && F.y != F.z)
            TLR_CUDA_TRY(cudaMemcpyAsync(F.y, F.z, I.n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        I.gram = std::vector<DevBuf>(I.nt);
        I.vty = std::vector<DevBuf>(I.nt);
        I.gram_n.assign(I.nt, 0);
        I.gram_off.assign(I.nt, {});
        nt_max = std::max(nt_max, I.nt);
        items.push_back(std::move(it));
    }
    std::vector<cudaEvent_t> aux_marks;  // potrf + inverse on the side stream (profiling)
    // the side streams must not start before the buffers above exist
    TLR_CUDA_TRY(cudaEventRecord(ctx->ev_fork, st));
    TLR_CUDA_TRY(cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
    TLR_CUDA_TRY(cudaStreamWaitEvent(ctx->la, ctx->ev_fork, 0));
    TLR_CUDA_TRY(cudaStreamWaitEvent(ctx->sv, ctx->ev_fork, 0));
    // a compression job's tile belongs to items[J.item]
    const GrowSlot grow = [&](const CompressJob &J, int r, double **U, double **V) -> bool {
        const GrowSlot &gs = items[(size_t)J.item]->grow;
        return gs && gs(J, r, U, V);
    };

    // stage boundary events (profiling): 6 marks per column
    std::vector<cudaEvent_t> marks;
    auto mark = [&]() {
        if (!ctx->profile) return;
        profile_events(ctx, prof_used + 1);
        cudaEvent_t e = ctx->prof_events[prof_used++];
        TLR_CUDA_TRY(cudaEventRecord(e, st));
        marks.push_back(e);
    };
    // detail marks (profiling): each attributes the time since the previous
    // mark on its stream to one of the kDetail buckets
    struct DMark {
        cudaEvent_t e;
        int idx;
    };
    std::vector<DMark> dm_main, dm_aux, dm_la, dm_sv;
    auto dmark = [&](std::vector<DMark> &v, cudaStream_t s, int idx) {
        if (!ctx->profile) return;
        profile_events(ctx, prof_used + 1);
        cudaEvent_t e = ctx->prof_events[prof_used++];
        TLR_CUDA_TRY(cudaEventRecord(e, s));
        v.push_back(DMark{e, idx});
    };
    // On an error the buffers above are released stream-ordered on st while
    // the side and look-ahead streams may still use them: wait for those first.
    struct SideStreamGuard {
        tlr_ctx *ctx;
        ~SideStreamGuard() {
            if (std::uncaught_exceptions()) {
                cudaStreamSynchronize(ctx->sv);
                cudaStreamSynchronize(ctx->la);
                cudaStreamSynchronize(ctx->aux);
                cudaStreamSynchronize(ctx->hp);
            }
        }
    } side_guard{ctx};
    using Hold = std::vector<std::unique_ptr<DevBuf>>;
    auto hold_buf = [](Hold &h, size_t bytes, cudaStream_t s) -> DevBuf & {
        h.push_back(std::make_unique<DevBuf>(bytes, s));
        return *h.back();
    };

    // Update of column c's panel T (the tiles i >= c stacked, leading
    // dimension (nt - c) nb) by the factor columns k0 <= k < k1, for every
    // factorisation of `us` (panel buffer `buf`):
    //   T = A - P Q'  (generate: the Matern epilogue evaluates A)  or  T -= P Q',
    // with Q = [U_ck]_k and the P block (i, k) = U_ik W_ik, W_ik = V_ik' V_ck a
    // block of G_k.  A factorisation's panel is one GEMM and the GEMMs of all
    // of them share one launch; all work on stream s.
    auto panel_update = [&](const std::vector<GroupItem *> &us, int c, int k0, int k1, int buf, cudaStream_t s,
                            bool generate, std::vector<DMark> &dm, int det_build, int det_gemm, int ctas_per_sm) {
        Hold hold;
        std::vector<CopyDesc> cq;
        std::vector<GemmProb> gp, gbig;
        std::vector<SplitDesc> sd;
        std::vector<MaternItem> mitems;
        std::vector<std::pair<double *, size_t>> zero;
        for (GroupItem *u : us) {
            GroupItem &I = *u;
            tlr_mat *M = I.M;
            const int nb = I.nb, nt = I.nt;
            const int64_t n = I.n;
            FactorStats *stats = I.in->stats;
            const int mc = tile_rows(n, nb, c);
            const int64_t Mp = (int64_t)(nt - c) * nb;
            std::vector<int> off(std::max(k1 - k0, 0) + 1, 0);
            for (int k = k0; k < k1; ++k) off[k - k0 + 1] = off[k - k0] + I.r_of(c, k);
            const int Rc = off.back();
            double *Qc = hold_buf(hold, (size_t)nb * std::max(Rc, 1) * sizeof(double), s).as<double>();
            double *Pc = hold_buf(hold, (size_t)Mp * std::max(Rc, 1) * sizeof(double), s).as<double>();
            if (Rc > 0) {
                for (int k = k0; k < k1; ++k)
                    if (I.r_of(c, k) > 0)
                        cq.push_back(CopyDesc{Uslot(M, c, k), nb, Qc + (int64_t)off[k - k0] * nb, nb, mc, I.r_of(c, k)});
                zero.emplace_back(Pc, (size_t)Mp * Rc * sizeof(double));
                for (int k = k0; k < k1; ++k) {
                    const int rck = I.r_of(c, k);
                    if (rck <= 0) continue;
                    const int S = I.gram_n[k];
                    const double *Gk = I.gram[k].as<double>();
                    for (int i = c; i < nt; ++i) {
                        const int rik = I.r_of(i, k);
                        if (rik <= 0) continue;
                        GemmProb b{};
                        b.A = Uslot(M, i, k); b.lda = nb; b.m = tile_rows(n, nb, i); b.k = rik;
                        b.B = Gk + (int64_t)I.gram_off[k][c] * S + I.gram_off[k][i]; b.ldb = S; b.n = rck;
                        b.C = Pc + (int64_t)off[k - k0] * Mp + (int64_t)(i - c) * nb; b.ldc = (int)Mp;
                        gp.push_back(b);
                        stats->flops += 2.0 * b.m * rik * rck;
                    }
                }
            }
            const int64_t rows_valid = n - (int64_t)c * nb;
            GemmProb g{};
            g.A = Pc; g.lda = (int)Mp; g.m = (int)Mp; g.k = Rc;
            g.B = Qc; g.ldb = nb; g.n = mc;
            g.C = I.panel_buf[buf].as<double>(); g.ldc = (int)Mp;
            g.ri0 = (int64_t)c * nb; g.ci0 = (int64_t)c * nb;
            g.item = (int)mitems.size();
            mitems.push_back(MaternItem{I.in->xy, n, I.in->P ? *I.in->P : MaternParams{}});
            if (df && !tcp && Rc > 0) {
                float2 *p2 = hold_buf(hold, (size_t)Mp * Rc * sizeof(float2), s).as<float2>();
                float2 *q2 = hold_buf(hold, (size_t)nb * Rc * sizeof(float2), s).as<float2>();
                g.A2 = p2;
                g.B2 = q2;
                sd.push_back(SplitDesc{Pc, p2, (int)Mp, (int)Mp, Rc});
                sd.push_back(SplitDesc{Qc, q2, nb, mc, Rc});
            }
            gbig.push_back(g);
            if (generate) {
                stats->matern_entries += (double)rows_valid * mc;
                stats->panel_launches += 1;
            }
            stats->gemm_flops += 2.0 * (double)rows_valid * mc * Rc;
            stats->flops += 2.0 * (double)rows_valid * mc * Rc;
        }
        copy_batched(ctx, s, cq);
        for (auto &z : zero) TLR_CUDA_TRY(cudaMemsetAsync(z.first, 0, z.second, s));
        gemm_batched(ctx, s, false, false, gp, 1.0, 0.0);
        split_f2_batched(ctx, s, sd);
        dmark(dm, s, det_build);
        std::vector<GemmProb> prod;  // problems with an inner dimension
        for (const GemmProb &g : gbig)
            if (g.k > 0) prod.push_back(g);
        if (generate && tcp) {
            // the covariance panels by a plain FP64 kernel, then T -= P Q' on the
            // tensor cores: their CTAs stay short (the FP64 Matern evaluation
            // would keep a tensor-core CTA, its tensor memory and its shared
            // memory, on an SM ~100 us per tile)
            for (const GemmProb &g : gbig) {
                const MaternItem &mi = mitems[(size_t)g.item];
                generate_panel(mi.xy, mi.n, g.ri0, g.ci0, g.m, g.n, mi.P, g.C, g.ldc, s);
            }
            if (!prod.empty()) gemm_tc(ctx, s, false, true, prod, -1.0, 1.0, kTcSlicesDefault, ctas_per_sm > 0);
        } else if (generate && gbig.size() == 1) {
            const MaternItem &mi = mitems[0];
            gemm_batched_matern(ctx, s, true, gbig, -1.0, mi.xy, mi.n, mi.P, df, 0, ctas_per_sm);
        } else if (generate) {
            gemm_batched_matern_multi(ctx, s, gbig, -1.0, mitems, df, ctas_per_sm);
        } else if (!prod.empty() && tcp) {
            gemm_tc(ctx, s, false, true, prod, -1.0, 1.0);
        } else if (!prod.empty()) {
            gemm_batched(ctx, s, false, true, prod, -1.0, 1.0, df);
        }
        dmark(dm, s, det_gemm);
    };

    // Look-ahead correction of column c's panel by column k = c - 1 alone:
    //   T_ic -= U_ik Z_i,  Z_i = W_ik U_ck',  W_ik = V_ik' V_ck  (a block of G_k),
    // grouped so that the inner dimension of the large product is r_ik.
    auto panel_correct = [&](const std::vector<GroupItem *> &us, int c, int buf, cudaStream_t s) {
        Hold hold;
        std::vector<GemmProb> gz, gu;
        std::vector<SplitDesc> sd;
        for (GroupItem *u : us) {
            GroupItem &I = *u;
            tlr_mat *M = I.M;
            const int nb = I.nb, nt = I.nt;
            const int64_t n = I.n;
            FactorStats *stats = I.in->stats;
            double *T = I.panel_buf[buf].as<double>();
            const int k = c - 1;
            const int rck = I.r_of(c, k);
            if (rck <= 0) continue;
            const int mc = tile_rows(n, nb, c);
            const int64_t Mp = (int64_t)(nt - c) * nb;
            const int S = I.gram_n[k];
            const double *Gk = I.gram[k].as<double>();
            int64_t ztot = 0;
            std::vector<int64_t> zoff(nt, -1);
            for (int i = c; i < nt; ++i)
                if (I.r_of(i, k) > 0) {
                    zoff[i] = ztot;
                    ztot += I.r_of(i, k);
                }
            if (ztot == 0) continue;
            double *zb = hold_buf(hold, (size_t)ztot * nb * sizeof(double), s).as<double>();
            float2 *u2 = dfp ? hold_buf(hold, (size_t)ztot * nb * sizeof(float2), s).as<float2>() : nullptr;
            float2 *z2 = dfp ? hold_buf(hold, (size_t)ztot * nb * sizeof(float2), s).as<float2>() : nullptr;
            for (int i = c; i < nt; ++i) {
                const int rik = I.r_of(i, k);
                if (rik <= 0) continue;
                GemmProb a{};
                a.A = Gk + (int64_t)I.gram_off[k][c] * S + I.gram_off[k][i]; a.lda = S; a.m = rik; a.k = rck;
                a.B = Uslot(M, c, k); a.ldb = nb; a.n = mc;
                a.C = zb + zoff[i] * nb; a.ldc = rik;
                gz.push_back(a);
                GemmProb b{};
                b.A = Uslot(M, i, k); b.lda = nb; b.m = tile_rows(n, nb, i); b.k = rik;
                b.B = zb + zoff[i] * nb; b.ldb = rik; b.n = mc;
                b.C = T + (int64_t)(i - c) * nb; b.ldc = (int)Mp;
                if (dfp) {
                    const int64_t o = zoff[i] * nb;
                    sd.push_back(SplitDesc{b.A, u2 + o, nb, b.m, b.k});
                    sd.push_back(SplitDesc{b.B, z2 + o, b.k, b.k, mc});
                    b.A2 = u2 + o;
                    b.B2 = z2 + o;
                }
                gu.push_back(b);
                stats->flops += 2.0 * rik * rck * mc + 2.0 * b.m * rik * mc;
                stats->gemm_flops += 2.0 * b.m * rik * mc;
            }
        }
        gemm_batched(ctx, s, false, true, gz, 1.0, 0.0);
        split_f2_batched(ctx, s, sd);
        if (tcc) gemm_tc(ctx, s, false, false, gu, -1.0, 1.0);
        else gemm_batched(ctx, s, false, false, gu, -1.0, 1.0, df);
    };

    // y_c -= sum_{k<c} U_ck c_k, c_k = V_ck' y_k: a slice of column k's V_k' y_k
    auto solve_update = [&](const std::vector<GroupItem *> &us, int c, cudaStream_t ss) {
        Hold hold;
        std::vector<CopyDesc> cq, cc;
        std::vector<GemmProb> gg;
        for (GroupItem *u : us) {
            GroupItem &I = *u;
            tlr_mat *M = I.M;
            const int nb = I.nb;
            const int mc = tile_rows(I.n, nb, c);
            std::vector<int> off(c + 1, 0);
            for (int k = 0; k < c; ++k) off[k + 1] = off[k] + I.r_of(c, k);
            const int Rc = off[c];
            if (Rc <= 0) continue;
            double *qb = hold_buf(hold, (size_t)nb * Rc * sizeof(double), ss).as<double>();
            double *cb = hold_buf(hold, (size_t)Rc * sizeof(double), ss).as<double>();
            for (int k = 0; k < c; ++k) {
                const int r = I.r_of(c, k);
                if (r <= 0) continue;
                cq.push_back(CopyDesc{Uslot(M, c, k), nb, qb + (int64_t)off[k] * nb, nb, mc, r});
                cc.push_back(CopyDesc{I.vty[k].as<double>() + I.gram_off[k][c], r, cb + off[k], r, r, 1});
            }
            GemmProb g{};
            g.A = qb; g.lda = nb; g.m = mc; g.k = Rc;
            g.B = cb; g.ldb = Rc; g.n = 1;
            g.C = I.in->y + (int64_t)c * nb; g.ldc = nb;
            gg.push_back(g);
        }
        copy_batched(ctx, ss, cq);
        copy_batched(ctx, ss, cc);
        gemm_batched(ctx, ss, false, false, gg, -1.0, 1.0);
    };

    // status words of the call: one per factorisation (the context's word
    // itself for a single one), after the context's word
    const bool own_words = G > 1;
    auto status_of = [&](const GroupItem &I) { return own_words ? ctx->d_status + 1 + I.idx : ctx->d_status; };
    auto fail = [&](GroupItem &I, int code, long long info, const std::string &msg) {
        I.active = false;
        I.in->err = code;
        I.in->msg = msg;
        *I.in->info = info;
    };

    int cur = 0;
    bool sv_pending = false;  // a solve on the solve stream may still read X
    for (int j = 0; j < nt_max; ++j) {
        std::vector<GroupItem *> act;
        for (auto &u : items)
            if (u->active && j < u->nt) act.push_back(u.get());
        if (act.empty()) break;
        mark();
        dmark(dm_main, st, -1);
        // --- panel: T_{:,j} = A_{:,j} - sum_{k<j} L_{:,k} L_jk'
        std::vector<GroupItem *> fresh, corr;
        for (GroupItem *u : act) (u->ahead && j > 0 ? corr : fresh).push_back(u);
        if (!fresh.empty()) {
            if (mode == FactorMode::Tlr) {
                // densify the compressed input column: T_jj = D_jj, T_ij = U_ij V_ij'
                GroupItem &I = *fresh[0];
                tlr_mat *M = I.M;
                const int nb = I.nb, nt = I.nt, mj = tile_rows(I.n, nb, j);
                const int64_t Mp = (int64_t)(nt - j) * nb;
                double *Tp = I.panel_buf[cur].as<double>();
                TLR_CUDA_TRY(cudaMemsetAsync(Tp, 0, (size_t)Mp * nb * sizeof(double), st));
                copy_batched(ctx, st, {CopyDesc{M->D + (int64_t)j * nb * nb, nb, Tp, (int)Mp, mj, mj}});
                std::vector<GemmProb> gd;
                for (int i = j + 1; i < nt; ++i) {
                    int rin = I.prev[(size_t)i * nt + j];
                    if (rin <= 0) continue;
                    GemmProb a{};
                    a.A = Uslot(M, i, j); a.lda = nb; a.m = tile_rows(I.n, nb, i); a.k = rin;
                    a.B = Vslot(M, i, j); a.ldb = nb; a.n = mj;
                    a.C = Tp + (int64_t)(i - j) * nb; a.ldc = (int)Mp;
                    gd.push_back(a);
                }
                gemm_batched(ctx, st, false, true, gd, 1.0, 0.0);
            }
            panel_update(fresh, j, 0, j, cur, st, mode == FactorMode::Matern, dm_main, kDetBuild, kDetPanel, 0);
        }
        if (!corr.empty()) {
            // the update by the columns k < j - 1 ran on the look-ahead stream
            TLR_CUDA_TRY(cudaStreamWaitEvent(st, ctx->ev_la_join, 0));
            dmark(dm_main, st, kDetAheadWait);
            panel_correct(corr, j, cur, st);
            dmark(dm_main, st, kDetCorrect);
        }
        mark();
        if (dfp) {
            std::vector<SplitDesc> sd;
            for (GroupItem *u : act)
                if (j + 1 < u->nt) {
                    const int64_t Mp = (int64_t)(u->nt - j) * u->nb;
                    sd.push_back(SplitDesc{u->panel_buf[cur].as<double>() + u->nb, u->Tp2 + u->nb, (int)Mp,
                                           (int)(Mp - u->nb), tile_rows(u->n, u->nb, j)});
                }
            if (!sd.empty()) {
                split_f2_batched(ctx, st, sd);
                dmark(dm_main, st, kDetSplit);
            }
        }
        mark();
        // --- L_jj = chol(T_jj) into D_j and X = L_jj^-1, on the side stream:
        // they are independent of the compression of the column's other tiles
        {
            std::vector<CopyDesc> cd;
            std::vector<PotrfJob> pj;
            for (GroupItem *u : act) {
                const int nb = u->nb, mj = tile_rows(u->n, nb, j);
                const int64_t Mp = (int64_t)(u->nt - j) * nb;
                double *Dj = u->M->D + (int64_t)j * nb * nb;
                cd.push_back(CopyDesc{u->panel_buf[cur].as<double>(), (int)Mp, Dj, nb, mj, mj});
                pj.push_back(PotrfJob{Dj, nb, mj, u->Xinv, nb, nullptr, status_of(*u), (long long)j * nb});
                u->in->stats->flops += (double)mj * mj * mj / 3.0 + (double)mj * mj * mj / 3.0;
            }
            copy_batched(ctx, st, cd);
            TLR_CUDA_TRY(cudaEventRecord(ctx->ev_fork, st));
            TLR_CUDA_TRY(cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
            // the previous column's solve reads X = L^-1 on the solve stream
            if (sv_pending) TLR_CUDA_TRY(cudaStreamWaitEvent(ctx->aux, ctx->ev_sv_done, 0));
            if (ctx->profile) {
                profile_events(ctx, prof_used + 1);
                TLR_CUDA_TRY(cudaEventRecord(ctx->prof_events[prof_used], ctx->aux));
                aux_marks.push_back(ctx->prof_events[prof_used++]);
            }
            dmark(dm_aux, ctx->aux, -1);
            potrf_inv_batched(ctx, ctx->aux, pj, df);  // one cluster launch per column of the group
            dmark(dm_aux, ctx->aux, kDetPotrf);
            if (ctx->profile) {
                profile_events(ctx, prof_used + 1);
                TLR_CUDA_TRY(cudaEventRecord(ctx->prof_events[prof_used], ctx->aux));
                aux_marks.push_back(ctx->prof_events[prof_used++]);
            }
            TLR_CUDA_TRY(cudaEventRecord(ctx->ev_join, ctx->aux));
        }
        // --- look-ahead: column j+1's update by the columns k < j, concurrently
        // with this column's compression (G_k, k < j, are final)
        {
            std::vector<GroupItem *> la;
            for (GroupItem *u : act)
                if (u->ahead && j + 1 < u->nt) la.push_back(u);
            if (!la.empty()) {
                TLR_CUDA_TRY(cudaEventRecord(ctx->ev_la_fork, st));
                TLR_CUDA_TRY(cudaStreamWaitEvent(ctx->la, ctx->ev_la_fork, 0));
                dmark(dm_la, ctx->la, -1);
                panel_update(la, j + 1, 0, j, cur ^ 1, ctx->la, true, dm_la, kDetAheadBuild, kDetAheadPanel,
                             ahead_ctas);
                TLR_CUDA_TRY(cudaEventRecord(ctx->ev_la_join, ctx->la));
            }
        }
        mark();
        // --- compress T_ij, i > j, of every factorisation (main stream,
        // concurrently with the above); one launch per class serves them all
        std::vector<CompressJob> jobs;
        std::vector<std::pair<GroupItem *, int>> job_of;  // (factorisation, tile row)
        for (GroupItem *u : act) {
            const int nb = u->nb, nt = u->nt;
            const int64_t Mp = (int64_t)(nt - j) * nb;
            double *Tp = u->panel_buf[cur].as<double>();
            for (int i = j + 1; i < nt; ++i) {
                CompressJob c{};
                c.T = Tp + (int64_t)(i - j) * nb;
                c.ldt = (int)Mp;
                c.T2 = dfp ? u->Tp2 + (int64_t)(i - j) * nb : nullptr;
                c.m = tile_rows(u->n, nb, i);
                c.k = tile_rows(u->n, nb, j);
                c.U = Uslot(u->M, i, j);
                c.ldu = nb;
                c.V = Vslot(u->M, i, j);
                c.ldv = nb;
                c.s_guess = u->have_prev ? u->prev[(size_t)i * nt + j] : 32;
                c.tile_id = (long long)i * nt + j;
                c.cap = slot_cap(u->M, i, j);
                c.tau = u->in->tau;
                c.maxrank = u->M->maxrank;
                c.item = u->idx;
                jobs.push_back(c);
                job_of.emplace_back(u, i);
            }
        }
        std::vector<int> rk, fails;
        dmark(dm_main, st, kDetDiagCopy);
        // the status words ride on the compression's own host read of its
        // ranks: its first round waits for the side stream's POTRF and copies
        // them, so that a tile column syncs the host once, not twice
        const int nwords = own_words ? G + 1 : 1;
        bool have_status = false;
        const std::function<void()> read_status = [&]() {
            TLR_CUDA_TRY(cudaStreamWaitEvent(ctx->hp, ctx->ev_join, 0));
            TLR_CUDA_TRY(cudaMemcpyAsync(ctx->h_status, ctx->d_status, nwords * sizeof(DevStatus),
                                         cudaMemcpyDeviceToHost, ctx->hp));
            have_status = true;
        };
        if (!jobs.empty()) {
            // on the high-priority stream, ahead of the look-ahead GEMM
            TLR_CUDA_TRY(cudaEventRecord(ctx->ev_hp_fork, st));
            TLR_CUDA_TRY(cudaStreamWaitEvent(ctx->hp, ctx->ev_hp_fork, 0));
            compress_jobs(ctx, ctx->hp, jobs, rk, fails, df, read_status, grow, tcc);
            TLR_CUDA_TRY(cudaEventRecord(ctx->ev_hp_join, ctx->hp));
            TLR_CUDA_TRY(cudaStreamWaitEvent(st, ctx->ev_hp_join, 0));
        }
        mark();
        dmark(dm_main, st, kDetCompress);
        TLR_CUDA_TRY(cudaStreamWaitEvent(st, ctx->ev_join, 0));
        dmark(dm_main, st, kDetJoin);
        // --- outcomes: the status words (read with the ranks above, or here
        // for a column with nothing to compress), then non-finite tiles, then
        // ranks that do not fit
        if (!have_status) {
            TLR_CUDA_TRY(cudaMemcpyAsync(ctx->h_status, ctx->d_status, nwords * sizeof(DevStatus),
                                         cudaMemcpyDeviceToHost, st));
            TLR_CUDA_TRY(cudaStreamSynchronize(st));
        }
        if (own_words && ctx->h_status[0].code)  // a device-wide failure (bounded wait ran out)
            throw make_error(ctx->h_status[0].code, "TLR Cholesky: device status %d", ctx->h_status[0].code);
        for (GroupItem *u : act) {
            const DevStatus &w = ctx->h_status[own_words ? 1 + u->idx : 0];
            if (w.code == TLR_ERR_NOT_SPD)
                fail(*u, w.code, w.info, make_error(w.code, "TLR Cholesky: non-positive pivot at row %lld", w.info).msg);
            else if (w.code)
                fail(*u, w.code, w.info, make_error(w.code, "TLR Cholesky: device status %d", w.code).msg);
        }
        for (int kind : {kCompNan, kCompBad})
            for (int q : fails) {
                GroupItem &I = *job_of[(size_t)q].first;
                if (!I.active || rk[(size_t)q] != kind) continue;
                const long long t = jobs[(size_t)q].tile_id, nt = I.nt;
                if (kind == kCompNan) {
                    fail(I, TLR_ERR_NAN, t, make_error(TLR_ERR_NAN, "tile (%lld, %lld) holds non-finite values", t / nt,
                                                       t % nt).msg);
                } else {
                    tlr_mat *M = I.M;
                    fail(I, TLR_ERR_RANK, t,
                         make_error(TLR_ERR_RANK, "tile (%lld, %lld) needs rank > %s %d", t / nt, t % nt,
                                    M->cap_overflow ? "its slot, and the overflow area is full:" : "maxrank",
                                    M->cap_overflow ? slot_cap(M, (int)(t / nt), (int)(t % nt)) : M->maxrank).msg);
                }
            }
        std::vector<GroupItem *> ok;
        for (GroupItem *u : act)
            if (u->active) ok.push_back(u);
        for (size_t q = 0; q < jobs.size(); ++q) {
            GroupItem &I = *job_of[q].first;
            if (!I.active) continue;
            const int i = job_of[q].second, nt = I.nt;
            I.M->h_ranks[(size_t)i * nt + j] = I.M->h_ranks[(size_t)j * nt + i] = rk[q];
            double m = jobs[q].m, k = jobs[q].k;
            I.in->stats->flops += 8.0 * m * k * (rk[q] + 8);  // sampling + projection GEMMs (approx.)
        }
        // --- V_ij <- L_jj^-1 V_ij as one batched GEMM into a scratch panel, then copied back
        {
            Hold hold;
            std::vector<GemmProb> gt, gg, gs, gv;
            std::vector<CopyDesc> cb;
            std::vector<SplitDesc> sd, sg;
            for (GroupItem *u : ok) {
                GroupItem &I = *u;
                tlr_mat *M = I.M;
                const int nb = I.nb, nt = I.nt, mj = tile_rows(I.n, nb, j);
                FactorStats *stats = I.in->stats;
                int64_t off_c = 0;
                for (int i = j + 1; i < nt; ++i) off_c += I.r_of(i, j);
                // the packed V factors of column j, alive through the solve step
                I.vtmp.alloc((size_t)nb * std::max<int64_t>(off_c, 1) * sizeof(double), st);
                double *vt = I.vtmp.as<double>();
                float2 *x2 = nullptr, *v2 = nullptr;
                if (dfp && off_c > 0) {
                    // paired-FP32 operands: X, and the V factors packed like the output
                    x2 = hold_buf(hold, (size_t)nb * nb * sizeof(float2), st).as<float2>();
                    v2 = hold_buf(hold, (size_t)nb * off_c * sizeof(float2), st).as<float2>();
                    sd.push_back(SplitDesc{I.Xinv, x2, nb, mj, mj});
                }
                off_c = 0;
                I.gram_off[j].assign(nt, -1);
                for (int i = j + 1; i < nt; ++i) {
                    int r = I.r_of(i, j);
                    if (r <= 0) continue;
                    I.gram_off[j][i] = (int)off_c;
                    GemmProb g{};
                    g.A = I.Xinv; g.lda = nb; g.m = mj; g.k = mj;
                    g.B = Vslot(M, i, j); g.ldb = nb; g.n = r;
                    g.C = vt + off_c * nb; g.ldc = nb;
                    if (dfp) {
                        const int64_t o = off_c * nb;
                        sd.push_back(SplitDesc{g.B, v2 + o, nb, mj, g.n});
                        g.A2 = x2;
                        g.B2 = v2 + o;
                    }
                    gt.push_back(g);
                    cb.push_back(CopyDesc{vt + off_c * nb, nb, Vslot(M, i, j), nb, mj, r});
                    off_c += r;
                    stats->flops += 2.0 * mj * mj * r;
                }
                // G_j = V_j' V_j for the later columns' updates
                const int S = (int)off_c;
                I.gram_n[j] = S;
                if (S > 0 && j + 1 < nt) {
                    I.gram[j].alloc((size_t)S * S * sizeof(double), st);
                    GemmProb g{};
                    g.A = vt; g.lda = nb; g.m = S; g.k = mj;
                    g.B = vt; g.ldb = nb; g.n = S;
                    g.C = I.gram[j].as<double>(); g.ldc = S;
                    if (dfp && !tcg) {
                        float2 *w2 = hold_buf(hold, (size_t)nb * S * sizeof(float2), st).as<float2>();
                        sg.push_back(SplitDesc{vt, w2, nb, mj, S});
                        g.A2 = g.B2 = w2;
                    }
                    gg.push_back(g);
                    stats->flops += 2.0 * S * S * mj;
                }
                if (I.solve && S > 0 && j + 1 < nt) I.vty[j].alloc((size_t)S * sizeof(double), st);
            }
            split_f2_batched(ctx, st, sd);
            if (tcc) gemm_tc(ctx, st, false, false, gt, 1.0, 0.0);
            else gemm_batched(ctx, st, false, false, gt, 1.0, 0.0, df);
            copy_batched(ctx, st, cb);
            dmark(dm_main, st, kDetTrsm);
            if (!gg.empty()) {
                split_f2_batched(ctx, st, sg);
                if (tcg) gemm_tc(ctx, st, true, false, gg, 1.0, 0.0);
                else gemm_batched(ctx, st, true, false, gg, 1.0, 0.0, df);
                dmark(dm_main, st, kDetGram);
            }
        }
        // --- the fused forward solve of column j on its own stream (a5), beside
        // the next column's panel correction and compression: y_j -= the
        // products with the earlier columns, y_j <- L_jj^-1 y_j, the
        // log-determinant and |y|^2 terms, and V_j' y_j for the later columns
        {
            std::vector<GroupItem *> sv;
            for (GroupItem *u : ok)
                if (u->solve) sv.push_back(u);
            if (!sv.empty()) {
                const cudaStream_t ss = ctx->sv;
                TLR_CUDA_TRY(cudaEventRecord(ctx->ev_sv_fork, st));
                TLR_CUDA_TRY(cudaStreamWaitEvent(ss, ctx->ev_sv_fork, 0));
                dmark(dm_sv, ss, -1);
                if (j > 0) {
                    solve_update(sv, j, ss);
                    dmark(dm_sv, ss, kDetSolveUpd);
                }
                std::vector<GemmProb> gy, gv;
                for (GroupItem *u : sv) {
                    const int nb = u->nb;
                    GemmProb g{};
                    g.A = u->Xinv; g.lda = nb; g.m = tile_rows(u->n, nb, j); g.k = g.m;
                    g.B = u->in->y + (int64_t)j * nb; g.ldb = nb; g.n = 1;
                    g.C = u->ytmp.as<double>(); g.ldc = nb;
                    gy.push_back(g);
                }
                gemm_batched(ctx, ss, false, false, gy, 1.0, 0.0);
                for (GroupItem *u : sv) {
                    const int nb = u->nb, nt = u->nt, mj = tile_rows(u->n, nb, j);
                    double *yj = u->in->y + (int64_t)j * nb, *acc = u->in->acc;
                    TLR_CUDA_TRY(cudaMemcpyAsync(yj, u->ytmp.as<double>(), mj * sizeof(double), cudaMemcpyDeviceToDevice, ss));
                    diag_logsum(ss, u->M->D + (int64_t)j * nb * nb, nb, mj, acc, status_of(*u), acc + 2);
                    sumsq(ss, yj, mj, acc + 1);
                    if (j + 1 < nt && u->gram_n[j] > 0)
                        for (int i = j + 1; i < nt; ++i) {
                            const int r = u->r_of(i, j);
                            if (r <= 0) continue;
                            GemmProb v{};  // the slice of V_j' y_j of tile (i, j)
                            v.A = Vslot(u->M, i, j); v.lda = nb; v.m = r; v.k = mj;
                            v.B = yj; v.ldb = nb; v.n = 1;
                            v.C = u->vty[j].as<double>() + u->gram_off[j][i]; v.ldc = r;
                            gv.push_back(v);
                        }
                }
                gemm_batched(ctx, ss, true, false, gv, 1.0, 0.0);
                dmark(dm_sv, ss, kDetSolve);
                TLR_CUDA_TRY(cudaEventRecord(ctx->ev_sv_done, ss));
                sv_pending = true;
            }
        }
        for (GroupItem *u : ok) u->vtmp.release();
        mark();
        if (mode == FactorMode::Matern) cur ^= 1;
    }
    // a factorisation that stopped may still have its look-ahead in flight;
    // the solve stream's last column
    TLR_CUDA_TRY(cudaEventRecord(ctx->ev_la_join, ctx->la));
    TLR_CUDA_TRY(cudaStreamWaitEvent(st, ctx->ev_la_join, 0));
    TLR_CUDA_TRY(cudaEventRecord(ctx->ev_sv_done, ctx->sv));
    TLR_CUDA_TRY(cudaStreamWaitEvent(st, ctx->ev_sv_done, 0));
    if (ctx->profile) {
        compress_profile_collect(ctx);
        for (std::vector<DMark> *v : {&dm_main, &dm_aux, &dm_la, &dm_sv})
            if (!v->empty()) TLR_CUDA_TRY(cudaEventSynchronize(v->back().e));
        for (std::vector<DMark> *v : {&dm_main, &dm_aux, &dm_la, &dm_sv})
            for (size_t k = 1; k < v->size(); ++k) {
                if ((*v)[k].idx < 0) continue;
                float ms = 0.f;
                TLR_CUDA_TRY(cudaEventElapsedTime(&ms, (*v)[k - 1].e, (*v)[k].e));
                pstats->detail_ms[(*v)[k].idx] += ms;
            }
    }
    for (auto &u : items)
        if (u->active) upload_ranks(u->M, st);
    if (ctx->profile) {
        // marks: 6 per column (start, after build, after panel, after potrf,
        // after compress, after trsm); panel interval = stage 1
        for (size_t c = 0; c + 5 < marks.size(); c += 6)
            for (int k = 0; k < kStages; ++k) {
                float ms = 0.f;
                TLR_CUDA_TRY(cudaEventElapsedTime(&ms, marks[c + k], marks[c + k + 1]));
                pstats->stage_ms[k] += ms;
            }
        pstats->stage_ms[2] = 0.f;
        for (size_t c = 0; c + 1 < aux_marks.size(); c += 2) {
            float ms = 0.f;
            TLR_CUDA_TRY(cudaEventElapsedTime(&ms, aux_marks[c], aux_marks[c + 1]));
            pstats->stage_ms[2] += ms;
        }
        pstats->gemm_ms += pstats->detail_ms[kDetPanel] + pstats->detail_ms[kDetAheadPanel];
    }
}

void factor(tlr_ctx *ctx, cudaStream_t st, tlr_mat *M, FactorMode mode, const double *xy,
            const MaternParams *P, double tau, FactorStats *stats, long long *info, const double *z,
            double *y, double *acc, bool df, bool tc) {
    std::vector<FactorItem> one(1);
    FactorItem &F = one[0];
    F.M = M; F.xy = xy; F.P = P; F.tau = tau; F.stats = stats; F.info = info;
    F.z = z; F.y = y; F.acc = acc;
    factor_group(ctx, st, one, mode, df, tc);
    if (F.err != TLR_OK) throw Error{F.err, F.msg};
}

// y = L^-1 z tile by tile; acc[0] += sum log L_ii, acc[1] += |y|^2.
void forward_solve(tlr_ctx *ctx, cudaStream_t st, const tlr_mat *M, const double *z, double *y,
                   double *acc) {
    const int nt = M->nt, nb = M->nb;
    const int64_t n = M->n;
    auto r_of = [&](int i, int k) { return (int)M->h_ranks[(size_t)i * nt + k]; };
    if (y != z) TLR_CUDA_TRY(cudaMemcpyAsync(y, z, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    int maxR = 0;
    for (int j = 0; j < nt; ++j) {
        int Rj = 0;
        for (int k = 0; k < j; ++k) Rj += r_of(j, k);
        maxR = std::max(maxR, Rj);
    }
    DevBuf cbuf((size_t)std::max(maxR, 1) * sizeof(double), st);
    double *c = cbuf.as<double>();
    for (int j = 0; j < nt; ++j) {
        const int mj = tile_rows(n, nb, j);
        double *yj = y + (int64_t)j * nb;
        std::vector<GemmProb> gc, gu;
        int o = 0;
        for (int k = 0; k < j; ++k) {
            int r = r_of(j, k);
            if (r <= 0) continue;
            GemmProb a{};  // c_k = V_jk' y_k
            a.A = Vslot(M, j, k); a.lda = nb; a.m = r; a.k = tile_rows(n, nb, k);
            a.B = y + (int64_t)k * nb; a.ldb = nb; a.n = 1;
            a.C = c + o; a.ldc = r;
            gc.push_back(a);
            o += r;
        }
        if (o > 0) {
            gemm_batched(ctx, st, true, false, gc, 1.0, 0.0);
            // y_j -= [U_j0 ...] c, accumulated one k at a time (distinct outputs per launch)
            o = 0;
            for (int k = 0; k < j; ++k) {
                int r = r_of(j, k);
                if (r <= 0) continue;
                GemmProb b{};
                b.A = Uslot(M, j, k); b.lda = nb; b.m = mj; b.k = r;
                b.B = c + o; b.ldb = r; b.n = 1;
                b.C = yj; b.ldc = nb;
                gemm_batched(ctx, st, false, false, std::vector<GemmProb>{b}, -1.0, 1.0);
                o += r;
            }
        }
        const double *Dj = M->D + (int64_t)j * nb * nb;
        trsm_left_lower(ctx, st, Dj, nb, mj, {RhsDesc{yj, 1, nb}});
        diag_logsum(st, Dj, nb, mj, acc, ctx->d_status);
        sumsq(st, yj, mj, acc + 1);
    }
}

// z = L w
void lmul(tlr_ctx *ctx, cudaStream_t st, const tlr_mat *M, const double *w, double *z) {
    const int nt = M->nt, nb = M->nb;
    const int64_t n = M->n;
    auto r_of = [&](int i, int k) { return (int)M->h_ranks[(size_t)i * nt + k]; };
    std::vector<GemmProb> gd;
    for (int i = 0; i < nt; ++i) {
        GemmProb a{};
        a.A = M->D + (int64_t)i * nb * nb; a.lda = nb; a.m = tile_rows(n, nb, i); a.k = a.m;
        a.B = w + (int64_t)i * nb; a.ldb = nb; a.n = 1;
        a.C = z + (int64_t)i * nb; a.ldc = nb;
        gd.push_back(a);
    }
    gemm_batched(ctx, st, false, false, gd, 1.0, 0.0);
    // c_ik = V_ik' w_k for all i > k
    int64_t tot = 0;
    std::vector<int64_t> co((size_t)nt * nt, -1);
    for (int i = 0; i < nt; ++i)
        for (int k = 0; k < i; ++k)
            if (r_of(i, k) > 0) { co[(size_t)i * nt + k] = tot; tot += r_of(i, k); }
    if (tot == 0) return;
    DevBuf cbuf((size_t)tot * sizeof(double), st);
    double *c = cbuf.as<double>();
    std::vector<GemmProb> gc;
    for (int i = 0; i < nt; ++i)
        for (int k = 0; k < i; ++k) {
            int r = r_of(i, k);
            if (r <= 0) continue;
            GemmProb a{};
            a.A = Vslot(M, i, k); a.lda = nb; a.m = r; a.k = tile_rows(n, nb, k);
            a.B = w + (int64_t)k * nb; a.ldb = nb; a.n = 1;
            a.C = c + co[(size_t)i * nt + k]; a.ldc = r;
            gc.push_back(a);
        }
    gemm_batched(ctx, st, true, false, gc, 1.0, 0.0);
    for (int k = 0; k < nt; ++k) {
        std::vector<GemmProb> gu;
        for (int i = k + 1; i < nt; ++i) {
            int r = r_of(i, k);
            if (r <= 0) continue;
            GemmProb b{};
            b.A = Uslot(M, i, k); b.lda = nb; b.m = tile_rows(n, nb, i); b.k = r;
            b.B = c + co[(size_t)i * nt + k]; b.ldb = r; b.n = 1;
            b.C = z + (int64_t)i * nb; b.ldc = nb;
            gu.push_back(b);
        }
        gemm_batched(ctx, st, false, false, gu, 1.0, 1.0);
    }
}

int64_t plan_slots(tlr_mat *M, const std::vector<int32_t> &hint) {
    const int nt = M->nt;
    const int64_t noff = (int64_t)nt * (nt - 1) / 2;
    M->base_off.clear();
    M->cap.clear();
    M->off.clear();
    M->cur_cap.clear();
    M->arena_off = M->arena_cols = M->arena_next = 0;
    if (hint.size() != (size_t)nt * nt) return std::max<int64_t>(noff, 1) * M->maxrank;
    M->base_off.resize((size_t)noff);
    M->cap.resize((size_t)noff);
    int64_t col = 0;
    for (int i = 1; i < nt; ++i)
        for (int j = 0; j < i; ++j) {
            const int r = std::max(0, (int)hint[(size_t)i * nt + j]);
            const int c = std::min(M->maxrank, (r + std::max(8, r / 4) + 7) & ~7);
            const int64_t k = off_index(i, j);
            M->base_off[(size_t)k] = col;
            M->cap[(size_t)k] = c;
            col += c;
        }
    M->arena_off = col;
    M->arena_cols = std::max<int64_t>(col / 8, 4 * (int64_t)M->maxrank);
    M->off = M->base_off;
    M->cur_cap = M->cap;
    return std::max<int64_t>(col + M->arena_cols, 1);
}

// Compress packed dense tiles (tlr_generate layout) into M.
void compress_packed(tlr_ctx *ctx, cudaStream_t st, const double *tiles, tlr_mat *M, double tau,
                     long long *info) {
    const int nt = M->nt, nb = M->nb;
    const int64_t n = M->n;
    std::vector<int32_t> prev = M->h_ranks;
    bool have_prev = prev.size() == (size_t)nt * nt;
    auto tile = [&](int i, int j) { return tiles + ((int64_t)i * (i + 1) / 2 + j) * nb * nb; };
    reset_slots(M);
    const GrowSlot grow = arena_grow(M);
    for (long long &v : ctx->comp_stats) v = 0;
    std::vector<CopyDesc> cd;
    for (int t = 0; t < nt; ++t)
        cd.push_back(CopyDesc{tile(t, t), nb, M->D + (int64_t)t * nb * nb, nb, nb, nb});
    copy_batched(ctx, st, cd);
    std::vector<CompressJob> jobs;
    for (int i = 0; i < nt; ++i)
        for (int j = 0; j < i; ++j) {
            CompressJob c{};
            c.T = tile(i, j); c.ldt = nb;
            c.m = tile_rows(n, nb, i); c.k = tile_rows(n, nb, j);
            c.U = Uslot(M, i, j); c.ldu = nb;
            c.V = Vslot(M, i, j); c.ldv = nb;
            c.s_guess = have_prev ? prev[(size_t)i * nt + j] : 32;
            c.tile_id = (long long)i * nt + j;
            c.cap = slot_cap(M, i, j);
            jobs.push_back(c);
        }
    std::vector<int32_t> &R = M->h_ranks;
    R.assign((size_t)nt * nt, 0);
    for (int t = 0; t < nt; ++t) R[(size_t)t * nt + t] = tile_rows(n, nb, t);
    *info = -1;
    if (!jobs.empty()) {
        std::vector<int> rk;
        long long bad = -1, nan = -1;
        compress_tiles(ctx, st, jobs, tau, M->maxrank, rk, &bad, &nan, false, nullptr, grow);
        if (nan >= 0) {
            *info = nan;
            throw make_error(TLR_ERR_NAN, "tile (%lld, %lld) holds non-finite values", nan / nt, nan % nt);
        }
        if (bad >= 0) {
            *info = bad;
            throw make_error(TLR_ERR_RANK, "tile (%lld, %lld) needs rank > maxrank %d", bad / nt,
                             bad % nt, M->maxrank);
        }
        size_t q = 0;
        for (int i = 0; i < nt; ++i)
            for (int j = 0; j < i; ++j, ++q) R[(size_t)i * nt + j] = R[(size_t)j * nt + i] = rk[q];
    }
    upload_ranks(M, st);
}

}  // namespace tlr
