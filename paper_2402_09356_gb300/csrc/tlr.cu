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

#include "common.cuh"
#include "compress.cuh"
#include "dense.cuh"
#include "gemm.cuh"
#include "matern.cuh"
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

static inline double *Uslot(tlr_mat *M, int i, int j) {
    return M->U + off_index(i, j) * (int64_t)M->nb * M->maxrank;
}
static inline double *Vslot(tlr_mat *M, int i, int j) {
    return M->V + off_index(i, j) * (int64_t)M->nb * M->maxrank;
}
static inline const double *Uslot(const tlr_mat *M, int i, int j) {
    return M->U + off_index(i, j) * (int64_t)M->nb * M->maxrank;
}
static inline const double *Vslot(const tlr_mat *M, int i, int j) {
    return M->V + off_index(i, j) * (int64_t)M->nb * M->maxrank;
}

void upload_ranks(tlr_mat *M, cudaStream_t s) {
    TLR_CUDA_TRY(cudaStreamSynchronize(s));
    TLR_CUDA_TRY(cudaMemcpy(M->ranks, M->h_ranks.data(), M->h_ranks.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice));
}

void factor(tlr_ctx *ctx, cudaStream_t st, tlr_mat *M, FactorMode mode, const double *xy,
            const MaternParams *P, double tau, FactorStats *stats, long long *info, const double *z,
            double *y, double *acc, bool df) {
    if (df && mode != FactorMode::Matern) throw make_error(TLR_ERR_ARG, "paired-FP32 products need the Matern mode");
    const int nt = M->nt, nb = M->nb;
    const int64_t n = M->n;
    *info = -1;
    std::vector<int32_t> &R = M->h_ranks;  // r_ij of the factor, filled column by column
    std::vector<int32_t> prev = R;         // previous ranks (input ranks for FactorMode::Tlr)
    bool have_prev = !prev.empty() && prev.size() == (size_t)nt * nt;
    if (mode == FactorMode::Tlr && !have_prev) throw make_error(TLR_ERR_ARG, "matrix holds no compressed input");
    int prof_used = 0;
    for (double &v : ctx->comp_ms) v = 0.0;
    for (long long &v : ctx->comp_stats) v = 0;
    R.assign((size_t)nt * nt, 0);
    for (int t = 0; t < nt; ++t) R[(size_t)t * nt + t] = tile_rows(n, nb, t);
    auto r_of = [&](int i, int k) { return (int)R[(size_t)i * nt + k]; };
    DevBuf panel((size_t)nt * nb * nb * sizeof(double), st);
    double *Tp = panel.as<double>();
    // paired-FP32 copy of the panel (mixed precision): operand of the compression products
    DevBuf panel2(df ? (size_t)nt * nb * nb * sizeof(float2) : 0, st);
    float2 *Tp2 = panel2.as<float2>();
    DevBuf xinv((size_t)nb * nb * sizeof(double), st);
    double *Xinv = xinv.as<double>();
    // fused forward solve (a5): y = L^-1 z column by column
    const bool solve = (z != nullptr && y != nullptr && acc != nullptr);
    DevBuf ytmp(solve ? (size_t)nb * sizeof(double) : 0, st);
    if (solve && y != z) TLR_CUDA_TRY(cudaMemcpyAsync(y, z, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    std::vector<cudaEvent_t> aux_marks;  // potrf + inverse on the side stream (profiling)
    // the side stream must not start before the buffers above exist
    TLR_CUDA_TRY(cudaEventRecord(ctx->ev_fork, st));
    TLR_CUDA_TRY(cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));

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
    std::vector<DMark> dm_main, dm_aux;
    // per finished column k: the Gram matrix G_k = V_k' V_k of its packed V
    // factors V_k = [V_ik]_{i>k} (order of i, zero-rank tiles left out), the
    // column offset of each tile in V_k, and V_k' y_k for the fused solve
    std::vector<DevBuf> gram(nt), vty(nt);
    std::vector<int> gram_n(nt, 0);
    std::vector<std::vector<int>> gram_off(nt);
    auto dmark = [&](std::vector<DMark> &v, cudaStream_t s, int idx) {
        if (!ctx->profile) return;
        profile_events(ctx, prof_used + 1);
        cudaEvent_t e = ctx->prof_events[prof_used++];
        TLR_CUDA_TRY(cudaEventRecord(e, s));
        v.push_back(DMark{e, idx});
    };
    for (int j = 0; j < nt; ++j) {
        const int mj = tile_rows(n, nb, j);
        const int64_t Mp = (int64_t)(nt - j) * nb;  // panel leading dimension
        mark();
        dmark(dm_main, st, -1);
        // --- Q_j = [U_j0 | ... ] and offsets
        std::vector<int> off(j + 1, 0);
        for (int k = 0; k < j; ++k) off[k + 1] = off[k] + r_of(j, k);
        const int Rj = off[j];
        DevBuf qbuf((size_t)nb * std::max(Rj, 1) * sizeof(double), st);
        DevBuf pbuf((size_t)Mp * std::max(Rj, 1) * sizeof(double), st);
        double *Qj = qbuf.as<double>(), *Pj = pbuf.as<double>();
        if (Rj > 0) {
            std::vector<CopyDesc> cq;
            for (int k = 0; k < j; ++k)
                if (r_of(j, k) > 0)
                    cq.push_back(CopyDesc{Uslot(M, j, k), nb, Qj + (int64_t)off[k] * nb, nb, mj, r_of(j, k)});
            copy_batched(ctx, st, cq);
            TLR_CUDA_TRY(cudaMemsetAsync(Pj, 0, (size_t)Mp * Rj * sizeof(double), st));
            dmark(dm_main, st, kDetBuildCopy);
            // P block (i, k) = U_ik W_ik with W_ik = V_ik' V_jk, a block of the
            // Gram matrix G_k of column k's V factors (formed once per column)
            std::vector<GemmProb> gp;
            for (int k = 0; k < j; ++k) {
                const int rjk = r_of(j, k);
                if (rjk <= 0) continue;
                const int S = gram_n[k];
                const double *G = gram[k].as<double>();
                for (int i = j; i < nt; ++i) {
                    const int rik = r_of(i, k);
                    if (rik <= 0) continue;
                    GemmProb b{};
                    b.A = Uslot(M, i, k); b.lda = nb; b.m = tile_rows(n, nb, i); b.k = rik;
                    b.B = G + (int64_t)gram_off[k][j] * S + gram_off[k][i]; b.ldb = S; b.n = rjk;
                    b.C = Pj + (int64_t)off[k] * Mp + (int64_t)(i - j) * nb; b.ldc = (int)Mp;
                    gp.push_back(b);
                    stats->flops += 2.0 * b.m * rik * rjk;
                }
            }
            gemm_batched(ctx, st, false, false, gp, 1.0, 0.0);
            dmark(dm_main, st, kDetBuildP);
        }
        if (solve && Rj > 0) {
            // y_j -= Q_j c, c_k = V_jk' y_k: a slice of column k's V' y_k
            DevBuf cb((size_t)Rj * sizeof(double), st);
            std::vector<CopyDesc> cc;
            for (int k = 0; k < j; ++k) {
                int r = r_of(j, k);
                if (r <= 0) continue;
                cc.push_back(CopyDesc{vty[k].as<double>() + gram_off[k][j], r, cb.as<double>() + off[k], r, r, 1});
            }
            copy_batched(ctx, st, cc);
            GemmProb g{};
            g.A = Qj; g.lda = nb; g.m = mj; g.k = Rj;
            g.B = cb.as<double>(); g.ldb = Rj; g.n = 1;
            g.C = y + (int64_t)j * nb; g.ldc = nb;
            gemm_batched(ctx, st, false, false, std::vector<GemmProb>{g}, -1.0, 1.0);
            dmark(dm_main, st, kDetBuildSolve);
        }
        mark();
        // --- panel: T_{:,j} = A_{:,j} - P_j Q_j'
        const int64_t rows_valid = n - (int64_t)j * nb;
        if (mode == FactorMode::Matern) {
            GemmProb g{};
            g.A = Pj; g.lda = (int)Mp; g.m = (int)Mp; g.k = Rj;
            g.B = Qj; g.ldb = nb; g.n = mj;
            g.C = Tp; g.ldc = (int)Mp;
            g.ri0 = (int64_t)j * nb; g.ci0 = (int64_t)j * nb;
            DevBuf p2(df ? (size_t)Mp * std::max(Rj, 1) * sizeof(float2) : 0, st);
            DevBuf q2(df ? (size_t)nb * std::max(Rj, 1) * sizeof(float2) : 0, st);
            if (df && Rj > 0) {
                g.A2 = p2.as<float2>();
                g.B2 = q2.as<float2>();
                split_f2_batched(ctx, st, {SplitDesc{Pj, p2.as<float2>(), (int)Mp, (int)Mp, Rj},
                                           SplitDesc{Qj, q2.as<float2>(), nb, mj, Rj}});
                dmark(dm_main, st, kDetSplit);
            }
            gemm_batched_matern(ctx, st, true, std::vector<GemmProb>{g}, -1.0, xy, n, *P, df);
            dmark(dm_main, st, kDetPanel);
            if (df && j + 1 < nt) {
                split_f2_batched(ctx, st, {SplitDesc{Tp + nb, Tp2 + nb, (int)Mp, (int)(Mp - nb), mj}});
                dmark(dm_main, st, kDetSplit);
            }
            stats->gemm_flops += 2.0 * (double)rows_valid * mj * Rj;
            stats->matern_entries += (double)rows_valid * mj;
            stats->panel_launches += 1;
        } else {
            // densify the compressed input column: T_jj = D_jj, T_ij = U_ij V_ij'
            TLR_CUDA_TRY(cudaMemsetAsync(Tp, 0, (size_t)Mp * nb * sizeof(double), st));
            copy_batched(ctx, st, {CopyDesc{M->D + (int64_t)j * nb * nb, nb, Tp, (int)Mp, mj, mj}});
            std::vector<GemmProb> gd;
            for (int i = j + 1; i < nt; ++i) {
                int rin = prev[(size_t)i * nt + j];
                if (rin <= 0) continue;
                GemmProb a{};
                a.A = Uslot(M, i, j); a.lda = nb; a.m = tile_rows(n, nb, i); a.k = rin;
                a.B = Vslot(M, i, j); a.ldb = nb; a.n = mj;
                a.C = Tp + (int64_t)(i - j) * nb; a.ldc = (int)Mp;
                gd.push_back(a);
            }
            gemm_batched(ctx, st, false, true, gd, 1.0, 0.0);
            if (Rj > 0) {
                GemmProb g{};
                g.A = Pj; g.lda = (int)Mp; g.m = (int)Mp; g.k = Rj;
                g.B = Qj; g.ldb = nb; g.n = mj;
                g.C = Tp; g.ldc = (int)Mp;
                gemm_batched(ctx, st, false, true, std::vector<GemmProb>{g}, -1.0, 1.0);
            }
            stats->gemm_flops += 2.0 * (double)rows_valid * mj * Rj;
        }
        stats->flops += 2.0 * (double)rows_valid * mj * Rj;
        mark();
        // --- L_jj = chol(T_jj) into D_j and X = L_jj^-1, on the side stream:
        // they are independent of the compression of the column's other tiles
        double *Dj = M->D + (int64_t)j * nb * nb;
        copy_batched(ctx, st, {CopyDesc{Tp, (int)Mp, Dj, nb, mj, mj}});
        TLR_CUDA_TRY(cudaEventRecord(ctx->ev_fork, st));
        TLR_CUDA_TRY(cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
        // the side stream's launches go first: its chain of small dependent
        // kernels then starts before the compression fills the GPU
        auto enqueue_aux = [&]() {
            if (ctx->profile) {
                profile_events(ctx, prof_used + 1);
                TLR_CUDA_TRY(cudaEventRecord(ctx->prof_events[prof_used], ctx->aux));
                aux_marks.push_back(ctx->prof_events[prof_used++]);
            }
            dmark(dm_aux, ctx->aux, -1);
            potrf_dense(ctx, ctx->aux, Dj, nb, mj, (long long)j * nb);
            dmark(dm_aux, ctx->aux, kDetPotrf);
            set_identity(ctx->aux, Xinv, nb, mj);
            trsm_left_lower(ctx, ctx->aux, Dj, nb, mj, {RhsDesc{Xinv, mj, nb}});
            dmark(dm_aux, ctx->aux, kDetInverse);
            if (ctx->profile) {
                profile_events(ctx, prof_used + 1);
                TLR_CUDA_TRY(cudaEventRecord(ctx->prof_events[prof_used], ctx->aux));
                aux_marks.push_back(ctx->prof_events[prof_used++]);
            }
            TLR_CUDA_TRY(cudaEventRecord(ctx->ev_join, ctx->aux));
        };
        enqueue_aux();
        stats->flops += (double)mj * mj * mj / 3.0 + (double)mj * mj * mj / 3.0;
        mark();
        // --- compress T_ij, i > j (main stream, concurrently with the above)
        std::vector<CompressJob> jobs;
        for (int i = j + 1; i < nt; ++i) {
            CompressJob c{};
            c.T = Tp + (int64_t)(i - j) * nb;
            c.ldt = (int)Mp;
            c.T2 = df ? Tp2 + (int64_t)(i - j) * nb : nullptr;
            c.m = tile_rows(n, nb, i);
            c.k = mj;
            c.U = Uslot(M, i, j);
            c.ldu = nb;
            c.V = Vslot(M, i, j);
            c.ldv = nb;
            c.s_guess = have_prev ? prev[(size_t)i * nt + j] : 32;
            c.tile_id = (long long)i * nt + j;
            jobs.push_back(c);
        }
        std::vector<int> rk;
        long long bad = -1, nan = -1;
        dmark(dm_main, st, kDetDiagCopy);
        if (!jobs.empty()) compress_tiles(ctx, st, jobs, tau, M->maxrank, rk, &bad, &nan, df);
        mark();
        dmark(dm_main, st, kDetCompress);
        TLR_CUDA_TRY(cudaStreamWaitEvent(st, ctx->ev_join, 0));
        dmark(dm_main, st, kDetJoin);
        long long sinfo = -1;
        int sc = status_fetch(ctx, st, &sinfo);  // syncs st, after the side stream's work
        if (sc) { *info = sinfo; throw make_error(sc, "TLR Cholesky: non-positive pivot at row %lld", sinfo); }
        if (nan >= 0) {
            *info = nan;
            throw make_error(TLR_ERR_NAN, "tile (%lld, %lld) holds non-finite values", nan / nt, nan % nt);
        }
        if (bad >= 0) {
            *info = bad;
            throw make_error(TLR_ERR_RANK, "tile (%lld, %lld) needs rank > maxrank %d", bad / nt, bad % nt,
                             M->maxrank);
        }
        for (size_t q = 0; q < jobs.size(); ++q) {
            int i = j + 1 + (int)q;
            R[(size_t)i * nt + j] = R[(size_t)j * nt + i] = rk[q];
            double m = jobs[q].m, k = jobs[q].k;
            stats->flops += 8.0 * m * k * (rk[q] + 8);  // sampling + projection GEMMs (approx.)
        }
        // --- V_ij <- L_jj^-1 V_ij as one batched GEMM into a scratch panel, then copied back
        DevBuf vtmp;  // the packed V factors of column j, alive through the solve step
        const double *vty_src = nullptr;
        int vty_pending = 0;
        {
            std::vector<GemmProb> gt;
            std::vector<CopyDesc> cb;
            int64_t off_c = 0;
            for (int i = j + 1; i < nt; ++i) off_c += r_of(i, j);
            vtmp.alloc((size_t)nb * std::max<int64_t>(off_c, 1) * sizeof(double), st);
            off_c = 0;
            gram_off[j].assign(nt, -1);
            for (int i = j + 1; i < nt; ++i) {
                int r = r_of(i, j);
                if (r <= 0) continue;
                gram_off[j][i] = (int)off_c;
                GemmProb g{};
                g.A = Xinv; g.lda = nb; g.m = mj; g.k = mj;
                g.B = Vslot(M, i, j); g.ldb = nb; g.n = r;
                g.C = vtmp.as<double>() + off_c * nb; g.ldc = nb;
                gt.push_back(g);
                cb.push_back(CopyDesc{vtmp.as<double>() + off_c * nb, nb, Vslot(M, i, j), nb, mj, r});
                off_c += r;
                stats->flops += 2.0 * mj * mj * r;
            }
            DevBuf x2(df && !gt.empty() ? (size_t)nb * nb * sizeof(float2) : 0, st);
            DevBuf v2(df && !gt.empty() ? (size_t)nb * std::max<int64_t>(off_c, 1) * sizeof(float2) : 0, st);
            if (df && !gt.empty()) {
                // paired-FP32 operands: X, and the V factors packed like the output
                std::vector<SplitDesc> sd{SplitDesc{Xinv, x2.as<float2>(), nb, mj, mj}};
                for (GemmProb &g : gt) {
                    const int64_t o = g.C - vtmp.as<double>();
                    sd.push_back(SplitDesc{g.B, v2.as<float2>() + o, nb, mj, g.n});
                    g.A2 = x2.as<float2>();
                    g.B2 = v2.as<float2>() + o;
                }
                split_f2_batched(ctx, st, sd);
            }
            gemm_batched(ctx, st, false, false, gt, 1.0, 0.0, df);
            copy_batched(ctx, st, cb);
            dmark(dm_main, st, kDetTrsm);
            // G_j = V_j' V_j for the later columns' updates
            const int S = (int)off_c;
            gram_n[j] = S;
            if (S > 0 && j + 1 < nt) {
                gram[j].alloc((size_t)S * S * sizeof(double), st);
                GemmProb g{};
                g.A = vtmp.as<double>(); g.lda = nb; g.m = S; g.k = mj;
                g.B = vtmp.as<double>(); g.ldb = nb; g.n = S;
                g.C = gram[j].as<double>(); g.ldc = S;
                DevBuf v2(df ? (size_t)nb * S * sizeof(float2) : 0, st);
                if (df) {
                    split_f2_batched(ctx, st, {SplitDesc{vtmp.as<double>(), v2.as<float2>(), nb, mj, S}});
                    g.A2 = g.B2 = v2.as<float2>();
                }
                gemm_batched(ctx, st, true, false, std::vector<GemmProb>{g}, 1.0, 0.0, df);
                stats->flops += 2.0 * S * S * mj;
                dmark(dm_main, st, kDetGram);
            }
            if (solve && S > 0 && j + 1 < nt) {
                // V_j' y_j once y_j is final (after the solve step below)
                vty[j].alloc((size_t)S * sizeof(double), st);
                vty_src = vtmp.as<double>();
                vty_pending = S;
            }
        }
        if (solve) {
            double *yj = y + (int64_t)j * nb;
            GemmProb g{};
            g.A = Xinv; g.lda = nb; g.m = mj; g.k = mj;
            g.B = yj; g.ldb = nb; g.n = 1;
            g.C = ytmp.as<double>(); g.ldc = nb;
            gemm_batched(ctx, st, false, false, std::vector<GemmProb>{g}, 1.0, 0.0);
            TLR_CUDA_TRY(cudaMemcpyAsync(yj, ytmp.as<double>(), mj * sizeof(double), cudaMemcpyDeviceToDevice, st));
            diag_logsum(st, Dj, nb, mj, acc, ctx->d_status);
            sumsq(st, yj, mj, acc + 1);
            if (vty_pending > 0) {
                GemmProb v{};
                v.A = vty_src; v.lda = nb; v.m = vty_pending; v.k = mj;
                v.B = yj; v.ldb = nb; v.n = 1;
                v.C = vty[j].as<double>(); v.ldc = vty_pending;
                gemm_batched(ctx, st, true, false, std::vector<GemmProb>{v}, 1.0, 0.0);
            }
            dmark(dm_main, st, kDetSolve);
        }
        mark();
    }
    if (ctx->profile) {
        for (std::vector<DMark> *v : {&dm_main, &dm_aux})
            if (!v->empty()) TLR_CUDA_TRY(cudaEventSynchronize(v->back().e));
        for (std::vector<DMark> *v : {&dm_main, &dm_aux})
            for (size_t k = 1; k < v->size(); ++k) {
                if ((*v)[k].idx < 0) continue;
                float ms = 0.f;
                TLR_CUDA_TRY(cudaEventElapsedTime(&ms, (*v)[k - 1].e, (*v)[k].e));
                stats->detail_ms[(*v)[k].idx] += ms;
            }
    }
    upload_ranks(M, st);
    if (ctx->profile) {
        // marks: 6 per column (start, after build, after panel, after potrf,
        // after compress, after trsm); panel interval = stage 1
        for (size_t c = 0; c + 5 < marks.size(); c += 6)
            for (int k = 0; k < kStages; ++k) {
                float ms = 0.f;
                TLR_CUDA_TRY(cudaEventElapsedTime(&ms, marks[c + k], marks[c + k + 1]));
                stats->stage_ms[k] += ms;
            }
        stats->stage_ms[2] = 0.f;
        for (size_t c = 0; c + 1 < aux_marks.size(); c += 2) {
            float ms = 0.f;
            TLR_CUDA_TRY(cudaEventElapsedTime(&ms, aux_marks[c], aux_marks[c + 1]));
            stats->stage_ms[2] += ms;
        }
        stats->gemm_ms += stats->stage_ms[1];
    }
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

// Compress packed dense tiles (tlr_generate layout) into M.
void compress_packed(tlr_ctx *ctx, cudaStream_t st, const double *tiles, tlr_mat *M, double tau,
                     long long *info) {
    const int nt = M->nt, nb = M->nb;
    const int64_t n = M->n;
    std::vector<int32_t> prev = M->h_ranks;
    bool have_prev = prev.size() == (size_t)nt * nt;
    auto tile = [&](int i, int j) { return tiles + ((int64_t)i * (i + 1) / 2 + j) * nb * nb; };
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
            jobs.push_back(c);
        }
    std::vector<int32_t> &R = M->h_ranks;
    R.assign((size_t)nt * nt, 0);
    for (int t = 0; t < nt; ++t) R[(size_t)t * nt + t] = tile_rows(n, nb, t);
    *info = -1;
    if (!jobs.empty()) {
        std::vector<int> rk;
        long long bad = -1, nan = -1;
        compress_tiles(ctx, st, jobs, tau, M->maxrank, rk, &bad, &nan);
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
