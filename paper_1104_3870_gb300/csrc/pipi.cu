// Two-pion correlators of total isospin I = 0, 1, 2 at zero total momentum (Sec. III two-meson
// diagrams, Sec. V two-pion operators): every Wick contraction of the four pion bilinears, each
// quark propagator replaced by a stochastic LapH line estimate (Sec. II), evaluated as traces of
// products of meson functions in dilution space.
//
// Operators.  A pion of momentum p at the sink is c_{ab} Phi_p[n, n'] qbar^A(t,a,n) q^B(t,b,n'),
// c = gamma_4 gamma_5, with (A, B) from the isospin triplet pi+ = ubar d, pi0 = (dbar d - ubar u)/sqrt 2,
// pi- = -dbar u; the two-pion state |I, I3> couples a pion of momentum p and one of -p with the
// Clebsch-Gordan coefficients of 1 x 1.  The source partner of the sink bilinear (c, Phi, A, B)
// is conj(c_{ab}) Phi_{-p}[n, n'] qbar^B(t0,b,n) q^A(t0,a,n') and its weight is conjugated.
//
// Wick's theorem.  With the four bilinears B_0, B_1 (sink, t_F) and B_2, B_3 (source, t_0),
//   < B_0 B_1 B_2 B_3 > = sum_sigma sgn(sigma) prod_{cycles} tr(M_k Q_k M_{sigma k} Q_{sigma k} ...),
// where Q_k is the propagator from the antiquark of B_{sigma k} to the quark of B_k and sigma runs
// over the permutations whose flavours match (quark of B_k = antiquark of B_{sigma k}).  The value
// of a permutation does not depend on the flavour labels, so the weights of all flavour terms are
// summed per permutation first and each permutation is evaluated once.
//
// Lines (Sec. II, the graphical rules of Sec. III).  A propagator whose antiquark end is a source
// bilinear takes a forward line sourced at t0, Q = sum_b phi^[b] rho^[b]dag; one from a sink
// bilinear to a source bilinear takes a forward line through gamma_5 Hermiticity,
// Q = G' (sum_b phi^[b] rho^[b]dag)^dag G' with G' = gamma_4 gamma_5; one between two sink
// bilinears takes a same-time line (every projector solved).  The lines of a term carry
// different noises: its propagators take the next unused forward (four) or same-time (two) line
// in the order the cycles are visited (cycles started from the lowest unvisited bilinear).  The
// rule is applied by the bilinear's side, so at t_F = t_0 a sink bilinear still takes the
// gamma_5-swapped or same-time lines.
//
// Dilution space.  With Q_s = X_s Y_s^dag, a cycle (k_0, ..., k_{L-1}) gives
//   tr(M_{k0} Q_0 ... M_{k_{L-1}} Q_{L-1}) = tr(F_0 F_1 ... F_{L-1}),  F_s = Y_{s-1}^dag M_{k_s} X_s,
// a meson function in the dilution indices of the lines on either side: X = phi (forward,
// same-time) or G' rho (swapped), Y = rho (forward, same-time) or G'^dag phi (swapped).  Sink
// F's are formed for every t_F at once.  Same-time lines are kept per slice: at t only the
// projectors whose time support holds t contribute, so those are gathered first.  All FP64.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "gamma_host.cuh"

namespace laph {

namespace {

enum LineKind { FWD = 0, BWD = 1, SMT = 2 };

// Same-time line gathered per slice: phi[t][j] = coef[bidx[t][j]][t], rho[t][j] = the diluted
// noise of projector bidx[t][j] on slice t ([nt][nbt][4][nv] each); bidx indexes the line's
// projector list (its coefficients and its masks).
__global__ void smt_gather_kernel(int nt, int nbt, int nv, const int *__restrict__ bidx, const c64 *__restrict__ coef,
                                  const uint8_t *__restrict__ codes, const uint8_t *__restrict__ mask,
                                  c64 *__restrict__ phi, c64 *__restrict__ rho) {
    const int t = blockIdx.x, j = blockIdx.y;
    const int b = bidx[t * nbt + j];
    const uint8_t *m = mask + (long)b * (nt + 4 + nv);
    for (int e = threadIdx.x; e < 4 * nv; e += blockDim.x) {
        const int a = e / nv, n = e % nv;
        phi[((long)t * nbt + j) * 4 * nv + e] = coef[((long)b * nt + t) * 4 * nv + e];
        c64 v{0, 0};
        if (m[t] && m[nt + a] && m[nt + 4 + n]) {
            const int code = codes[(t * 4 + a) * nv + n];
            v = code == 0 ? c64{1, 0} : code == 1 ? c64{0, 1} : code == 2 ? c64{-1, 0} : c64{0, -1};
        }
        rho[((long)t * nbt + j) * 4 * nv + e] = v;
    }
}

// out[t][b][a][n] = sum_m Phi[tp][n][m] in(b, t)[a][m] with in(b, t) at in + b sb + t st and
// tp = t (sink) or t1 (one source slice); out compact [T][nb][4][nv].
__global__ void phi_strided_kernel(int nv, int nb, int t1, int sink, const c64 *__restrict__ phi,
                                   const c64 *__restrict__ in, long sb, long st, c64 *__restrict__ out) {
    const int b = blockIdx.x, t = blockIdx.y;
    const c64 *f = phi + (long)(sink ? t : t1) * nv * nv;
    const c64 *src = in + (long)b * sb + (long)t * st;
    c64 *dst = out + ((long)t * nb + b) * 4 * nv;
    for (int e = threadIdx.x; e < 4 * nv; e += blockDim.x) {
        const int a = e / nv, n = e % nv;
        c64 s{0, 0};
        for (int m = 0; m < nv; ++m) s += f[(long)n * nv + m] * src[a * nv + m];
        dst[e] = s;
    }
}

// F[t][b1][b2] = sum_{n} sum_{a,b} conj(A(b1, t)[a][n]) W[a][b] B(b2, t)[b][n], strided operands
__global__ void mfn_kernel(int nbA, int nbB, int nv, const c64 *__restrict__ A, long sbA, long stA,
                           const c64 *__restrict__ B, long sbB, long stB, W4 W, c64 *__restrict__ F) {
    extern __shared__ c64 aw[];   // [4][nv]
    const int t = blockIdx.x, b1 = blockIdx.y;
    const c64 *a = A + (long)b1 * sbA + (long)t * stA;
    for (int e = threadIdx.x; e < 4 * nv; e += blockDim.x) {
        const int bb = e / nv, n = e % nv;
        c64 s{0, 0};
#pragma unroll
        for (int al = 0; al < 4; ++al) s += conj(a[al * nv + n]) * W.w[al][bb];
        aw[e] = s;
    }
    __syncthreads();
    for (int b2 = threadIdx.x; b2 < nbB; b2 += blockDim.x) {
        const c64 *bp = B + (long)b2 * sbB + (long)t * stB;
        c64 s{0, 0};
        for (int e = 0; e < 4 * nv; ++e) s += aw[e] * bp[e];
        F[((long)t * nbA + b1) * nbB + b2] = s;
    }
}

// C[t] = A[t or 0] B[t or 0], A [m][k], B [k][n]
__global__ void bmm_kernel(int m, int k, int n, const c64 *__restrict__ A, long sA, const c64 *__restrict__ B, long sB,
                           c64 *__restrict__ C) {
    const int t = blockIdx.x, i = blockIdx.y;
    const c64 *a = A + t * sA + (long)i * k;
    const c64 *b = B + t * sB;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        c64 s{0, 0};
        for (int l = 0; l < k; ++l) s += a[l] * b[(long)l * n + j];
        C[((long)t * m + i) * n + j] = s;
    }
}

// tr[t] = sum_{i<m, j<n} A[t][i][j] B[t][j][i]  (B = nullptr: tr A[t], m = n)
__global__ void trprod_kernel(int m, int n, const c64 *__restrict__ A, long sA, const c64 *__restrict__ B, long sB,
                              c64 *__restrict__ tr) {
    __shared__ c64 sm[256];
    const int t = blockIdx.x;
    const c64 *a = A + t * sA;
    c64 acc{0, 0};
    if (B == nullptr) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) acc += a[(long)i * n + i];
    } else {
        const c64 *b = B + t * sB;
        for (long e = threadIdx.x; e < (long)m * n; e += blockDim.x) {
            const long i = e / n, j = e % n;
            acc += a[e] * b[j * m + i];
        }
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) tr[t] = sm[0];
}

struct Traces {
    const c64 *tr[4];
    int per_t[4];
};

// corr[dt] += w prod_c tr_c[t_F or 0], t_F = (t0 + dt) mod nt
__global__ void term_accum_kernel(int nt, int t0, int ncyc, Traces T, c64 w, c64 *corr) {
    const int dt = blockIdx.x * blockDim.x + threadIdx.x;
    if (dt >= nt) return;
    const int tf = (t0 + dt) % nt;
    c64 v = w;
    for (int c = 0; c < ncyc; ++c) v = v * T.tr[c][T.per_t[c] ? tf : 0];
    corr[dt] += v;
}

// ---------------------------------------------------------------- host side: operators and Wick terms
struct Bil {
    int qbar, q;   // flavour labels: 0 = u, 1 = d
};
struct Term {
    double w;
    Bil b[2];
};

// pion triplet as (weight, (antiquark, quark)): pi+ = ubar d, pi0 = (dbar d - ubar u)/sqrt 2, pi- = -dbar u
static std::vector<std::pair<double, Bil>> pion_flavours(int m) {
    const double r = 1.0 / std::sqrt(2.0);
    if (m == 1) return {{1.0, {0, 1}}};
    if (m == 0) return {{-r, {0, 0}}, {r, {1, 1}}};
    return {{-1.0, {1, 0}}};
}

// Clebsch-Gordan coefficients <1 m1; 1 m2 | I I3> as (weight, m1, m2)
static std::vector<std::tuple<double, int, int>> cg_1x1(int I, int I3) {
    const double r2 = 1.0 / std::sqrt(2.0), r3 = 1.0 / std::sqrt(3.0), r6 = 1.0 / std::sqrt(6.0);
    if (I == 2 && I3 == 2) return {{1.0, 1, 1}};
    if (I == 2 && I3 == 1) return {{r2, 1, 0}, {r2, 0, 1}};
    if (I == 2 && I3 == 0) return {{r6, 1, -1}, {2.0 * r6, 0, 0}, {r6, -1, 1}};
    if (I == 1 && I3 == 1) return {{r2, 1, 0}, {-r2, 0, 1}};
    if (I == 1 && I3 == 0) return {{r2, 1, -1}, {-r2, -1, 1}};
    if (I == 0 && I3 == 0) return {{r3, 1, -1}, {-r3, 0, 0}, {r3, -1, 1}};
    return {};
}

// sink terms: flavours as written; source terms: each bilinear's partner swaps antiquark and quark
static std::vector<Term> two_pion_terms(int I, int I3, bool source) {
    std::vector<Term> out;
    for (auto &cg : cg_1x1(I, I3))
        for (auto &f1 : pion_flavours(std::get<1>(cg)))
            for (auto &f2 : pion_flavours(std::get<2>(cg))) {
                Term t;
                t.w = std::get<0>(cg) * f1.first * f2.first;
                t.b[0] = source ? Bil{f1.second.q, f1.second.qbar} : f1.second;
                t.b[1] = source ? Bil{f2.second.q, f2.second.qbar} : f2.second;
                out.push_back(t);
            }
    return out;
}

struct LineRef {
    int kind, idx;
};

}  // namespace

}  // namespace laph

using namespace laph;

extern "C" int correlate_pipi(laph_ctx *ctx, const laph_lattice *lat, const laph_pipi_spec *spec,
                              const void *const *coef_fwd, const uint8_t *const *noise_fwd, const void *const *coef_smt,
                              const uint8_t *const *noise_smt, const void *phi_p, const void *phi_mp, void *corr,
                              void *stream) {
    return guard([&] {
        ctx_activate(ctx);
        LAPH_REQUIRE(lat != nullptr && spec != nullptr && corr != nullptr, "null argument");
        const int nt = lat->nt, nv = spec->nv, t0 = spec->t0, nbf = spec->nb_fwd, nbs = spec->nb_smt;
        LAPH_REQUIRE(nt >= 1 && nv >= 1 && nbf >= 1 && nbf <= 4096 && nbs >= 0 && nbs <= 65535, "bad sizes");
        LAPH_REQUIRE(t0 >= 0 && t0 < nt, "t0 out of range");
        LAPH_REQUIRE(!cg_1x1(spec->iso, spec->iso3).empty(), "isospin (I, I3) must have 0 <= I <= 2, 0 <= I3 <= I");
        LAPH_REQUIRE((phi_p == nullptr) == (phi_mp == nullptr), "phi_p and phi_mp must both be given or both null");
        LAPH_REQUIRE(coef_fwd != nullptr && noise_fwd != nullptr && spec->b_fwd != nullptr, "null forward lines");
        cudaStream_t s = as_stream(stream);

        // weight of every permutation sigma: sum over sink x source flavour terms it contracts
        const std::vector<Term> snk = two_pion_terms(spec->iso, spec->iso3, false);
        const std::vector<Term> src = two_pion_terms(spec->iso, spec->iso3, true);
        std::vector<int> perm = {0, 1, 2, 3};
        std::vector<std::pair<std::vector<int>, double>> perms;
        do {
            double w = 0.0;
            for (const Term &a : snk)
                for (const Term &b : src) {
                    const Bil bl[4] = {a.b[0], a.b[1], b.b[0], b.b[1]};
                    bool ok = true;
                    for (int k = 0; k < 4; ++k) ok &= bl[k].q == bl[perm[k]].qbar;
                    if (ok) w += a.w * b.w;
                }
            if (std::fabs(w) > 1e-14) perms.push_back({perm, w});
        } while (std::next_permutation(perm.begin(), perm.end()));

        // line assignment per permutation (cycles in order, next unused line of each kind)
        struct Cycle {
            std::vector<int> k;
            std::vector<LineRef> q;   // q[s]: propagator from the antiquark of B_{sigma k_s} to the quark of B_{k_s}
        };
        struct Eval {
            std::vector<Cycle> cyc;
            double w;
            int sign;
        };
        std::vector<Eval> evals;
        bool need_smt = false;
        for (auto &pw : perms) {
            const std::vector<int> &pm = pw.first;
            Eval ev;
            ev.w = pw.second;
            int nf = 0, ns = 0, ncyc = 0;
            bool seen[4] = {false, false, false, false};
            for (int k0 = 0; k0 < 4; ++k0) {
                if (seen[k0]) continue;
                Cycle c;
                for (int k = k0; !seen[k]; k = pm[k]) {
                    seen[k] = true;
                    c.k.push_back(k);
                    const bool src_end = pm[k] >= 2, snk_end = k >= 2;   // antiquark end at t0 / quark end at t0
                    if (src_end) c.q.push_back({FWD, nf++});
                    else if (snk_end) c.q.push_back({BWD, nf++});
                    else c.q.push_back({SMT, ns++});
                }
                ev.cyc.push_back(c);
                ++ncyc;
            }
            ev.sign = ((4 - ncyc) % 2) ? -1 : 1;
            need_smt |= ns > 0;
            LAPH_REQUIRE(nf <= 4 && ns <= 2, "internal: line count");
            evals.push_back(ev);
        }

        // forward lines: sinks [nbf][nt][4][nv], noise at t0 [nbf][4][nv]
        std::vector<uint8_t> mf = dilution_masks(spec->dil_fwd, nt, nv, spec->b_fwd, nbf);
        uint8_t *dmf = (uint8_t *)ws_get(ctx, "pp:maskf", mf.size());
        LAPH_CUDA(cudaMemcpyAsync(dmf, mf.data(), mf.size(), cudaMemcpyHostToDevice, s));
        const size_t fbytes = sizeof(c64) * (size_t)nbf * nt * 4 * nv;
        const c64 *phf[4];
        c64 *rhf[4];
        for (int k = 0; k < 4; ++k) {
            LAPH_REQUIRE(coef_fwd[k] != nullptr && noise_fwd[k] != nullptr, "forward line arrays are null");
            const std::string id = std::to_string(k);
            phf[k] = (const c64 *)stage_in(ctx, coef_fwd[k], fbytes, "pp:cf" + id, s);
            const uint8_t *codes = (const uint8_t *)stage_in(ctx, noise_fwd[k], (size_t)nt * 4 * nv, "pp:nf" + id, s);
            rhf[k] = (c64 *)ws_get(ctx, "pp:rf" + id, sizeof(c64) * nbf * 4 * nv);
            rho_at_t0_kernel<<<grid_for((long)nbf * 4 * nv, 256), 256, 0, s>>>(nt, nv, nbf, t0, codes, dmf, rhf[k]);
            LAPH_LAUNCH_CHECK();
        }
        // same-time lines gathered per slice: [nt][nbt][4][nv]
        int nbt = 0;
        c64 *phs[2] = {nullptr, nullptr}, *rhs_[2] = {nullptr, nullptr};
        if (need_smt) {
            LAPH_REQUIRE(nbs >= 1 && spec->b_smt != nullptr && coef_smt != nullptr && noise_smt != nullptr,
                         "this isospin needs same-time lines");
            std::vector<uint8_t> ms = dilution_masks(spec->dil_smt, nt, nv, spec->b_smt, nbs);
            std::vector<int> bidx;
            for (int t = 0; t < nt; ++t) {
                int cnt = 0;
                for (int j = 0; j < nbs; ++j)
                    if (ms[(size_t)j * (nt + 4 + nv) + t]) {
                        bidx.push_back(j);
                        ++cnt;
                    }
                if (t == 0) nbt = cnt;
                LAPH_REQUIRE(cnt == nbt && cnt > 0,
                             "same-time lines: every slice must be covered by the same number of projectors");
            }
            uint8_t *dms = (uint8_t *)ws_get(ctx, "pp:masks", ms.size());
            LAPH_CUDA(cudaMemcpyAsync(dms, ms.data(), ms.size(), cudaMemcpyHostToDevice, s));
            int *dix = (int *)ws_get(ctx, "pp:bidx", sizeof(int) * bidx.size());
            LAPH_CUDA(cudaMemcpyAsync(dix, bidx.data(), sizeof(int) * bidx.size(), cudaMemcpyHostToDevice, s));
            for (int k = 0; k < 2; ++k) {
                LAPH_REQUIRE(coef_smt[k] != nullptr && noise_smt[k] != nullptr, "same-time line arrays are null");
                const std::string id = std::to_string(k);
                const c64 *cs = (const c64 *)stage_in(ctx, coef_smt[k], sizeof(c64) * (size_t)nbs * nt * 4 * nv,
                                                      "pp:cs" + id, s);
                const uint8_t *codes = (const uint8_t *)stage_in(ctx, noise_smt[k], (size_t)nt * 4 * nv, "pp:ns" + id, s);
                phs[k] = (c64 *)ws_get(ctx, "pp:ps" + id, sizeof(c64) * (size_t)nt * nbt * 4 * nv);
                rhs_[k] = (c64 *)ws_get(ctx, "pp:rs" + id, sizeof(c64) * (size_t)nt * nbt * 4 * nv);
                smt_gather_kernel<<<dim3(nt, nbt), 128, 0, s>>>(nt, nbt, nv, dix, cs, codes, dms, phs[k], rhs_[k]);
                LAPH_LAUNCH_CHECK();
            }
        }
        const c64 *dphi[2] = {nullptr, nullptr};
        if (phi_p != nullptr) {
            dphi[0] = (const c64 *)stage_in(ctx, phi_p, sizeof(c64) * (size_t)nt * nv * nv, "pp:phip", s);
            dphi[1] = (const c64 *)stage_in(ctx, phi_mp, sizeof(c64) * (size_t)nt * nv * nv, "pp:phim", s);
        }

        // operand views: pointer, strides, time dependence, dilution size
        struct View {
            const c64 *p;
            long sb, st;
            int nb;
        };
        const long sp = 4L * nv;
        // X side (quark end of bilinear k) of line q; sink bilinears are batched over t_F
        auto xview = [&](bool sink, LineRef q) -> View {
            if (q.kind == FWD) return sink ? View{phf[q.idx], nt * sp, sp, nbf} : View{phf[q.idx] + t0 * sp, nt * sp, 0, nbf};
            if (q.kind == BWD) return View{rhf[q.idx], sp, 0, nbf};
            return View{phs[q.idx], sp, nbt * sp, nbt};
        };
        // Y side (antiquark end)
        auto yview = [&](bool sink, LineRef q) -> View {
            if (q.kind == FWD) return View{rhf[q.idx], sp, 0, nbf};
            if (q.kind == BWD) return View{phf[q.idx], nt * sp, sink ? sp : 0, nbf};
            return View{rhs_[q.idx], sp, nbt * sp, nbt};
        };
        const Mat4 c = mat_mul(gamma_mat(3), gamma5());
        const Mat4 gp = c;   // G' = gamma_4 gamma_5
        const Mat4 Wk[4] = {c, c, mat_dag(c), mat_dag(c)};
        // bilinear k's momentum overlap: Phi_p, Phi_-p at the sink; Phi_-p, Phi_p at the source
        const int phik[4] = {0, 1, 1, 0};

        // F_s = Y^dag M_k X, cached per (k, Y line, X line); [T][nbY][nbX], T = nt (sink) or 1
        std::map<std::tuple<int, int, int, int, int>, std::pair<c64 *, int>> fcache;
        auto Fmat = [&](int k, LineRef y, LineRef x, int &nbY, int &nbX) -> c64 * {
            const bool sink = k < 2;
            const View vy = yview(sink, y), vx = xview(sink, x);
            nbY = vy.nb;
            nbX = vx.nb;
            auto key = std::make_tuple(k, y.kind, y.idx, x.kind, x.idx);
            auto it = fcache.find(key);
            if (it != fcache.end()) return it->second.first;
            const int T = sink ? nt : 1;
            View bx = vx;
            if (dphi[0] != nullptr) {   // Phi applied to the quark side first
                c64 *tmp = (c64 *)ws_get(ctx, "pp:phx", sizeof(c64) * (size_t)T * vx.nb * 4 * nv);
                phi_strided_kernel<<<dim3(vx.nb, T), 128, 0, s>>>(nv, vx.nb, t0, sink ? 1 : 0, dphi[phik[k]], vx.p,
                                                                  vx.sb, vx.st, tmp);
                LAPH_LAUNCH_CHECK();
                bx = View{tmp, sp, vx.nb * sp, vx.nb};
                if (!sink) bx.st = 0;
            }
            Mat4 W = Wk[k];
            if (y.kind == BWD) W = mat_mul(gp, W);   // Y = G'^dag phi: Y^dag = phi^dag G'
            if (x.kind == BWD) W = mat_mul(W, gp);   // X = G' rho
            char name[64];
            snprintf(name, sizeof name, "pp:F%d_%d_%d_%d_%d", k, y.kind, y.idx, x.kind, x.idx);
            c64 *F = (c64 *)ws_get(ctx, name, sizeof(c64) * (size_t)T * vy.nb * vx.nb);
            const int threads = vx.nb < 128 ? 128 : 256;
            mfn_kernel<<<dim3(T, vy.nb), threads, sizeof(c64) * 4 * nv, s>>>(vy.nb, vx.nb, nv, vy.p, vy.sb, vy.st, bx.p,
                                                                             bx.sb, bx.st, to_w4(W), F);
            LAPH_LAUNCH_CHECK();
            fcache[key] = {F, T};
            return F;
        };

        StagedOut out = stage_out(ctx, corr, sizeof(c64) * nt, "pp:corr");
        c64 *cdev = (c64 *)out.dev;
        LAPH_CUDA(cudaMemsetAsync(cdev, 0, sizeof(c64) * nt, s));
        for (const Eval &ev : evals) {
            Traces T{};
            int ci = 0;
            for (const Cycle &cy : ev.cyc) {
                const int L = (int)cy.k.size();
                std::vector<c64 *> f(L);
                std::vector<int> rows(L), cols(L), per_t(L);
                bool any_t = false;
                for (int sidx = 0; sidx < L; ++sidx) {
                    const LineRef y = cy.q[(sidx + L - 1) % L], x = cy.q[sidx];
                    f[sidx] = Fmat(cy.k[sidx], y, x, rows[sidx], cols[sidx]);
                    per_t[sidx] = cy.k[sidx] < 2;
                    any_t |= per_t[sidx] != 0;
                }
                const int Tc = any_t ? nt : 1;
                c64 *tr = (c64 *)ws_get(ctx, "pp:tr" + std::to_string(ci), sizeof(c64) * nt);
                // P = F_0 ... F_{L-2}, then tr(P F_{L-1})
                const c64 *P = f[0];
                long sP = per_t[0] ? (long)rows[0] * cols[0] : 0;
                for (int sidx = 1; sidx + 1 < L; ++sidx) {
                    c64 *Pn = (c64 *)ws_get(ctx, "pp:P" + std::to_string(sidx % 2),
                                            sizeof(c64) * (size_t)nt * rows[0] * cols[sidx]);
                    const long sF = per_t[sidx] ? (long)rows[sidx] * cols[sidx] : 0;
                    const int Tn = (sP != 0 || sF != 0) ? nt : 1;
                    bmm_kernel<<<dim3(Tn, rows[0]), 128, 0, s>>>(rows[0], cols[sidx - 1], cols[sidx], P, sP, f[sidx], sF,
                                                                 Pn);
                    LAPH_LAUNCH_CHECK();
                    P = Pn;
                    sP = Tn == nt ? (long)rows[0] * cols[sidx] : 0;
                }
                if (L == 1) {
                    trprod_kernel<<<Tc, 256, 0, s>>>(rows[0], cols[0], P, sP, nullptr, 0, tr);
                } else {
                    const long sF = per_t[L - 1] ? (long)rows[L - 1] * cols[L - 1] : 0;
                    trprod_kernel<<<Tc, 256, 0, s>>>(rows[0], cols[L - 2], P, sP, f[L - 1], sF, tr);
                }
                LAPH_LAUNCH_CHECK();
                T.tr[ci] = tr;
                T.per_t[ci] = any_t ? 1 : 0;
                ++ci;
            }
            term_accum_kernel<<<grid_for(nt, 256), 256, 0, s>>>(nt, t0, ci, T, c64{ev.w * ev.sign, 0.0}, cdev);
            LAPH_LAUNCH_CHECK();
        }
        out.commit(s);
        LAPH_CUDA(cudaStreamSynchronize(s));
    });
}
