// Pathwise adjoint of one interaction of the collision step (FP64, non-relativistic), for gradients of a loss of the
// final velocities with respect to the initial velocities, the weights and the Coulomb logarithm.
//
// Every random draw and every discrete decision of the step is held fixed: the Philox draws, the permutations and
// TA77 pairs, the accept test of the heavier particle (Sec. 3.2), the weight order, the energy-correction pass
// structure and the crossing pair (the one that absorbs the remainder of Delta E_s). Between those decisions the
// interaction is a smooth map  v_before -> v_after  with parameters w and lnL:
//   scatter  (Sec. 3.2, Eq. sab_TA77): s = kappa lnL w_max N_min / (mu^2 u^3), N97 A(s) from coth A - 1/A = e^-s or
//            TA77 delta = sqrt(s/2) g, the polar angle, the rotation of u, the lighter/heavier updates;
//   shift    (Eq. vp_pm): v_pm = v_ps - B w, B = sum m w (v_ps - v_bs) / sum m w^2;
//   Delta E  (Eq. Econs, Eq. DeltaEs): per-particle energy differences, split by mean weight x post-shift energy;
//   energy pairs (Eqs. vp1/vp2/vrel_inelastic, U_inelastic): capped pairs U = sign(D) fE K, the crossing pair
//            U = D - (sum of the earlier pairs' U); v1' = v1 + m2/M (g - 1) v_R, v2' = v2 - m1/M (g - 1) v_R,
//            g = sqrt(1 - U/K);
//   rollback (Sec. 5.2) when the correction fails: v_after = v_before.
// A Delta E_s that vanishes (equal weights, or below the rounding-noise threshold) is differentiated as its limit:
// the first pair of the order as the crossing pair with U = Delta E_s = 0.
// The kernel recomputes the interaction from the stored pre-interaction state, keeping a tape of every pair's inputs,
// then runs the chain rule backwards through the tape (one CTA per cell, the cell's working arrays in a per-CTA slab
// of the workspace). With a recorded tape the slabs are per cell and outlive the call: a recording call runs the
// forward and keeps each cell's slab (the tape and the per-cell scalars of the correction); a later replaying call on
// the same interaction runs only the reverse sweep from it.
#include "mcc_kernels.h"

namespace mcc {
namespace {

constexpr int kFlagTriplet = 1, kFlagUpdI = 2, kFlagUpdJ = 4, kFlagActive = 8;

struct AdjArgs {
    StepArgs a;                // state before the interaction (vx, vy, vz: double), w, constants of ic[0]
    double lnL;                // Coulomb logarithm of the interaction
    double* ox;                // state after the interaction (null: not written)
    double* oy;
    double* oz;
    double* gx;                // in: dL/dv after; out: dL/dv before (null: forward only)
    double* gy;
    double* gz;
    double* gw;                // += dL/dw
    double* glnL;              // += dL/dlnL (one value)
    char* slab;
    int64_t slab_stride;
    int32_t max_cell;
    int32_t max_epairs;
    int32_t tape;              // 0: per-CTA slabs, recompute; 1: per-cell slabs, record; 2: per-cell slabs, replay
};

// Per-cell scalars of the forward that the reverse sweep reads (kept at the end of a recorded slab).
struct TapeHead {
    int fail, ne[2], e0[2], zeroed[2];
    double B[3], Sw, S[3], dE, Es[2], W1[2], D[2];
};

// Per-CTA working arrays (n = max_cell, E = max_epairs).
struct Slab {
    uint64_t* keys;
    double* v;      // [3][n] working state
    double* vb;     // [3][n] before the interaction
    double* vp;     // [3][n] after the scatter
    double* vm;     // [3][n] after the momentum shift
    double* g;      // [3][n] gradient of the current stage
    double* gb;     // [3][n] gradient reaching v_before directly through the correction
    double* gwl;    // [n] dL/dw of this interaction
    double* pv;     // [6][n] per scatter pair: v_i, v_j at the pair's turn
    double* ev;     // [6][E] per energy pair: v_1, v_2 at the pair's turn
    double* eU;     // [E]
    double* eK;     // [E]
    int32_t* perm;  // [n] random permutation (cell-local indices, segment start included)
    int32_t* rho;   // [n] energy-pair order
    int32_t* pi;    // [n] scatter pair particles and flags
    int32_t* pj;
    int32_t* pf;
    int32_t* ei;    // [E] energy pair particles, capped flag
    int32_t* ej;
    int32_t* ecap;
    TapeHead* head;
    int n, E;
};

__host__ __device__ inline size_t al8(size_t x) { return (x + 7) & ~(size_t)7; }

__host__ __device__ inline size_t slab_bytes(int n, int E)
{
    const size_t dn = (size_t)n, de = (size_t)E;
    return al8(8 * dn) + 6 * al8(24 * dn) + al8(8 * dn) + al8(48 * dn) + al8(48 * de) + 2 * al8(8 * de) +
           5 * al8(4 * dn) + 3 * al8(4 * de) + al8(sizeof(TapeHead)) + 256;
}

__device__ Slab make_slab(char* base, int n, int E)
{
    Slab s;
    s.n = n;
    s.E = E;
    size_t o = 0;
    auto take = [&](size_t b) {
        char* p = base + o;
        o += al8(b);
        return p;
    };
    s.keys = reinterpret_cast<uint64_t*>(take(8 * (size_t)n));
    s.v = reinterpret_cast<double*>(take(24 * (size_t)n));
    s.vb = reinterpret_cast<double*>(take(24 * (size_t)n));
    s.vp = reinterpret_cast<double*>(take(24 * (size_t)n));
    s.vm = reinterpret_cast<double*>(take(24 * (size_t)n));
    s.g = reinterpret_cast<double*>(take(24 * (size_t)n));
    s.gb = reinterpret_cast<double*>(take(24 * (size_t)n));
    s.gwl = reinterpret_cast<double*>(take(8 * (size_t)n));
    s.pv = reinterpret_cast<double*>(take(48 * (size_t)n));
    s.ev = reinterpret_cast<double*>(take(48 * (size_t)E));
    s.eU = reinterpret_cast<double*>(take(8 * (size_t)E));
    s.eK = reinterpret_cast<double*>(take(8 * (size_t)E));
    s.perm = reinterpret_cast<int32_t*>(take(4 * (size_t)n));
    s.rho = reinterpret_cast<int32_t*>(take(4 * (size_t)n));
    s.pi = reinterpret_cast<int32_t*>(take(4 * (size_t)n));
    s.pj = reinterpret_cast<int32_t*>(take(4 * (size_t)n));
    s.pf = reinterpret_cast<int32_t*>(take(4 * (size_t)n));
    s.ei = reinterpret_cast<int32_t*>(take(4 * (size_t)E));
    s.ej = reinterpret_cast<int32_t*>(take(4 * (size_t)E));
    s.ecap = reinterpret_cast<int32_t*>(take(4 * (size_t)E));
    s.head = reinterpret_cast<TapeHead*>(take(sizeof(TapeHead)));
    return s;
}

struct AdjShared {
    int off[kMaxSpecies + 1];
    int fail;
    int ne[2];        // energy pairs taped per side
    int e0[2];        // first tape entry of each side
    int zeroed[2];    // Delta E_s set to zero as rounding noise
    double B[3], Sw, S[3];
    double dE, Es[2], W1[2], D[2], gD[2], gB[3];
    double gS[3], gSw, gdE, gEs[2], gW1[2];
    alignas(16) unsigned char red_raw[8 * kThreads * 8];
    alignas(8) unsigned char red[8 * 8];
};

__device__ __forceinline__ Acc<double>* accp(unsigned char* p) { return reinterpret_cast<Acc<double>*>(p); }

// Polar angle of one scatter pair with its derivatives: sin(Theta), 1 - cos(Theta) and d/ds of both.
__device__ void angle_and_derivative(const StepArgs& A, double s, double U1, double U4, double& st, double& omc,
                                     double& dst, double& domc)
{
    dst = 0.0;
    domc = 0.0;
    if (A.method == 0) {
        // TA77: delta = sqrt(s/2) g; both branches of the forward are sin = 2d/(1+d^2), 1-cos = 2d^2/(1+d^2)
        const double g = sqrt(-2.0 * log(U1)) * cospi(2.0 * U4);
        const double d = sqrt(0.5 * s) * g;
        const double den = 1.0 + d * d;
        st = 2.0 * d / den;
        omc = 2.0 * d * d / den;
        const double dd = s > 0.0 ? d / (2.0 * s) : 0.0;
        dst = 2.0 * (1.0 - d * d) / (den * den) * dd;
        domc = 4.0 * d / (den * den) * dd;
        return;
    }
    N97Tab<double> tab = {A.n97_f, A.n97_dh};
    const double Aa = n97_A(s, tab);
    double o, q;
    bool diff = true;
    if (Aa == 0.0) {
        o = 2.0 * U1;
        q = 2.0 * (1.0 - U1);
        diff = false;
    } else if (isinf(Aa)) {
        o = 0.0;
        q = 2.0;
        diff = false;
    } else {
        const double x = -U1 * -expm1(-2.0 * Aa);
        o = x > -0.5 ? -log1p(x) / Aa : -log((1.0 - U1) + U1 * exp(-2.0 * Aa)) / Aa;
        q = o <= 1.0 ? 2.0 - o : log1p((1.0 - U1) * expm1(2.0 * Aa)) / Aa;
    }
    bool co = false, cq = false;
    if (o < 0.0) { o = 0.0; co = true; }
    if (o > 2.0) { o = 2.0; co = true; }
    if (q < 0.0) { q = 0.0; cq = true; }
    if (q > 2.0) { q = 2.0; cq = true; }
    omc = o;
    st = sqrt(o * q);
    if (!diff) return;
    // 1 - cos = -ln Y / A with Y = (1 - U1) + U1 e^-2A; 1 + cos = 2 - (1 - cos)
    const double Y = (1.0 - U1) + U1 * exp(-2.0 * Aa);
    const double do_dA = co ? 0.0 : (-o / Aa + 2.0 * U1 * exp(-2.0 * Aa) / (Aa * Y));
    const double dq_dA = cq ? 0.0 : -(-o / Aa + 2.0 * U1 * exp(-2.0 * Aa) / (Aa * Y));
    // G(A) = 1 - (coth A - 1/A) = 1 - e^-s  =>  dA/ds = e^-s / G'(A)
    double G, dG;
    n97_G_dG(Aa, G, dG);
    const double dA_ds = exp(-s) / dG;
    domc = do_dA * dA_ds;
    dst = st > 0.0 ? (q * do_dA + o * dq_dA) / (2.0 * st) * dA_ds : 0.0;
}

// Forward of one scatter pair (the FP64 pair loop of the step kernel); returns the flags.
__device__ int pair_forward(const StepArgs& A, const InterConst& ic, double vi[3], double vj[3], double wi, double wj,
                            int nmin, bool trip, uint4 r)
{
    int flags = trip ? kFlagTriplet : 0;
    const double ux = vi[0] - vj[0], uy = vi[1] - vj[1], uz = vi[2] - vj[2];
    const double u2 = ux * ux + uy * uy + uz * uz;
    bool upd_i = true, upd_j = true;
    if (wi != wj) {
        const bool moves = u23<double>(r.z) * fmax(wi, wj) < fmin(wi, wj);
        if (wi > wj) upd_i = moves;
        else upd_j = moves;
    }
    if (upd_i) flags |= kFlagUpdI;
    if (upd_j) flags |= kFlagUpdJ;
    if (u2 == 0.0) return flags;
    flags |= kFlagActive;
    const double um = sqrt(u2);
    const double wmax = wi > wj ? wi : wj;
    double s = ic.kappa_mu2 * wmax * (double)nmin / (u2 * um);
    if (trip) s *= 0.5;
    double st, omc, dst, domc, sp, cp, d[3];
    angle_and_derivative(A, s, u23<double>(r.x), u23<double>(r.w), st, omc, dst, domc);
    sincospi(2.0 * u23<double>(r.y), &sp, &cp);
    rotate<double>(ux, uy, uz, st, omc, cp, sp, d[0], d[1], d[2]);
    for (int k = 0; k < 3; ++k) {
        if (upd_i) vi[k] += ic.mu_ma * d[k];
        if (upd_j) vj[k] -= ic.mu_mb * d[k];
    }
    return flags;
}

// Reverse of one scatter pair: g1, g2 (dL/d outputs) -> dL/d inputs in place; dL/dw of the heavier particle and
// dL/dlnL accumulated.
__device__ void pair_reverse(const StepArgs& A, const InterConst& ic, double lnL, const double vi[3],
                             const double vj[3], double wi, double wj, int nmin, int flags, uint4 r, double g1[3],
                             double g2[3], double& gwi, double& gwj, double& glnL)
{
    if (!(flags & kFlagActive)) return;
    const double fa = (flags & kFlagUpdI) ? ic.mu_ma : 0.0, fb = (flags & kFlagUpdJ) ? ic.mu_mb : 0.0;
    const double gd[3] = {fa * g1[0] - fb * g2[0], fa * g1[1] - fb * g2[1], fa * g1[2] - fb * g2[2]};
    if (gd[0] == 0.0 && gd[1] == 0.0 && gd[2] == 0.0) return;
    const double u[3] = {vi[0] - vj[0], vi[1] - vj[1], vi[2] - vj[2]};
    const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double um = sqrt(u2);
    const double wmax = wi > wj ? wi : wj;
    double s = ic.kappa_mu2 * wmax * (double)nmin / (u2 * um);
    if (flags & kFlagTriplet) s *= 0.5;
    double st, omc, dst, domc, sp, cp;
    angle_and_derivative(A, s, u23<double>(r.x), u23<double>(r.w), st, omc, dst, domc);
    sincospi(2.0 * u23<double>(r.y), &sp, &cp);
    // rotation du(u, st, omc) backwards
    double gst, gomc, gu[3];
    const double uperp = sqrt(u[0] * u[0] + u[1] * u[1]);
    double gum;
    if (uperp > 0.0) {
        const double a = u[0] / uperp, b = u[1] / uperp;
        gst = gd[0] * (a * u[2] * cp - b * um * sp) + gd[1] * (b * u[2] * cp + a * um * sp) - gd[2] * uperp * cp;
        gomc = -(gd[0] * u[0] + gd[1] * u[1] + gd[2] * u[2]);
        const double ga = gd[0] * u[2] * st * cp + gd[1] * um * st * sp;
        const double gb = -gd[0] * um * st * sp + gd[1] * u[2] * st * cp;
        gum = -gd[0] * b * st * sp + gd[1] * a * st * sp;
        double gup = -gd[2] * st * cp;
        gu[0] = -gd[0] * omc + ga / uperp;
        gu[1] = -gd[1] * omc + gb / uperp;
        gu[2] = gd[0] * a * st * cp + gd[1] * b * st * cp - gd[2] * omc;
        gup -= (ga * a + gb * b) / uperp;
        gu[0] += gup * a;
        gu[1] += gup * b;
    } else {
        gst = (gd[0] * cp + gd[1] * sp) * um;
        gomc = -gd[2] * u[2];
        gum = (gd[0] * cp + gd[1] * sp) * st;
        gu[0] = 0.0;
        gu[1] = 0.0;
        gu[2] = -gd[2] * omc;
    }
    // angle, then s = C w_max / um^3
    const double gs = gst * dst + gomc * domc;
    gum += gs * (-3.0 * s / um);
    for (int k = 0; k < 3; ++k) gu[k] += gum * u[k] / um;
    const double gwmax = gs * s / wmax;
    if (wi > wj) gwi += gwmax;
    else gwj += gwmax;
    glnL += gs * s / lnL;
    for (int k = 0; k < 3; ++k) {
        g1[k] += gu[k];
        g2[k] -= gu[k];
    }
}

__device__ __forceinline__ void ld3(const double* p, int n, int i, double x[3])
{
    x[0] = p[i];
    x[1] = p[n + i];
    x[2] = p[2 * n + i];
}
__device__ __forceinline__ void st3(double* p, int n, int i, const double x[3])
{
    p[i] = x[0];
    p[n + i] = x[1];
    p[2 * n + i] = x[2];
}

// k-th TA77 pair (cell-local indices) with p mod N_min supplied (inter).
__device__ __forceinline__ void pair_of(const Slab& sl, bool intra, int na, int nb, int a0, int b0, int p, int pm,
                                        int& i, int& j, bool& trip)
{
    trip = false;
    if (intra) {
        if (na & 1) {
            if (p < 3) {
                i = sl.perm[a0 + p];
                j = sl.perm[a0 + (p + 1) % 3];
                trip = true;
                return;
            }
            i = sl.perm[a0 + 2 * p - 3];
            j = sl.perm[a0 + 2 * p - 2];
            return;
        }
        i = sl.perm[a0 + 2 * p];
        j = sl.perm[a0 + 2 * p + 1];
        return;
    }
    if (na >= nb) {
        i = sl.perm[a0 + p];
        j = sl.perm[b0 + pm];
    } else {
        i = sl.perm[a0 + pm];
        j = sl.perm[b0 + p];
    }
}

__global__ void __launch_bounds__(kThreads) k_adjoint(const __grid_constant__ AdjArgs G)
{
    __shared__ AdjShared sh;
    const StepArgs& A = G.a;
    const InterConst& ic = A.ic[0];
    const int S = A.S;
    const bool intra = ic.a == ic.b;
    const double* wg = A.w;
    const double* gvx = reinterpret_cast<const double*>(A.vx);
    const double* gvy = reinterpret_cast<const double*>(A.vy);
    const double* gvz = reinterpret_cast<const double*>(A.vz);
    const uint32_t ictr = (uint32_t)A.inter_base;
    for (int c = blockIdx.x; c < A.n_cells; c += gridDim.x) {
        const Slab sl = make_slab(G.slab + (size_t)(G.tape ? c : (int)blockIdx.x) * (size_t)G.slab_stride, G.max_cell,
                                  G.max_epairs);
        const int64_t cs = A.offsets[(int64_t)c * S];
        const int n = (int)(A.offsets[(int64_t)(c + 1) * S] - cs);
        const int N = sl.n;
        if (n > N) {
            if (threadIdx.x == 0) latch(A.status, kErrBounds);
            continue;
        }
        if ((int)threadIdx.x <= S) sh.off[threadIdx.x] = (int)(A.offsets[(int64_t)c * S + threadIdx.x] - cs);
        for (int i = threadIdx.x; i < n; i += kThreads) {
            if (G.tape != 2) {  // a replaying call finds the state before the interaction in the tape
                const double x[3] = {gvx[cs + i], gvy[cs + i], gvz[cs + i]};
                st3(sl.v, N, i, x);
                st3(sl.vb, N, i, x);
            }
            sl.gwl[i] = 0.0;
        }
        __syncthreads();
        const int a0 = sh.off[ic.a], na = sh.off[ic.a + 1] - a0;
        const int b0 = sh.off[ic.b], nb = sh.off[ic.b + 1] - b0;
        const bool active = intra ? (na >= 2) : (na > 0 && nb > 0);
        const int nside = intra ? 1 : 2;
        if (active && G.tape == 2) {
            // ---- replay: the forward's per-cell scalars from the tape
            if (threadIdx.x == 0) {
                const TapeHead& h = *sl.head;
                sh.fail = h.fail;
                for (int k = 0; k < 2; ++k) {
                    sh.ne[k] = h.ne[k];
                    sh.e0[k] = h.e0[k];
                    sh.zeroed[k] = h.zeroed[k];
                    sh.Es[k] = h.Es[k];
                    sh.W1[k] = h.W1[k];
                    sh.D[k] = h.D[k];
                }
                for (int k = 0; k < 3; ++k) {
                    sh.B[k] = h.B[k];
                    sh.S[k] = h.S[k];
                }
                sh.Sw = h.Sw;
                sh.dE = h.dE;
            }
            __syncthreads();
        } else if (active) {
            // ---- forward: permutations (sorted Philox keys)
            for (int side = 0; side < nside; ++side) {
                const int s0 = side ? b0 : a0, ns = side ? nb : na;
                for (int q = threadIdx.x; q < ns; q += kThreads)
                    sl.keys[s0 + q] = perm_key(A.rng, (uint32_t)c, ictr, (uint32_t)side, (uint32_t)q);
                __syncthreads();
                block_sort_u64(sl.keys + s0, ns);
                for (int q = threadIdx.x; q < ns; q += kThreads) sl.perm[s0 + q] = s0 + (int)(sl.keys[s0 + q] & kPermMask);
                __syncthreads();
            }
            // ---- forward: scatter pairs in round order, inputs taped
            const int npairs = intra ? ((na & 1) ? (na + 3) / 2 : na / 2) : (na > nb ? na : nb);
            const int nmin = intra ? na - 1 : (na < nb ? na : nb);
            const int lead = (intra && (na & 1)) ? 3 : 0;
            const int round = intra ? npairs : nmin;
            for (int r0 = 0; r0 < npairs; r0 += round) {
                const int r1 = r0 + round < npairs ? r0 + round : npairs;
                int p = (lead && threadIdx.x == 0) ? 0 : r0 + lead + (int)threadIdx.x;
                while (p < r1) {
                    int i, j;
                    bool trip;
                    pair_of(sl, intra, na, nb, a0, b0, p, p - r0, i, j, trip);
                    double vi[3], vj[3];
                    ld3(sl.v, N, i, vi);
                    ld3(sl.v, N, j, vj);
                    for (int k = 0; k < 3; ++k) {
                        sl.pv[k * N + p] = vi[k];
                        sl.pv[(3 + k) * N + p] = vj[k];
                    }
                    const uint4 rr = draw(A.rng, (uint32_t)p, (uint32_t)c, ictr, kTagScat);
                    sl.pf[p] = pair_forward(A, ic, vi, vj, wg[cs + i], wg[cs + j], nmin, trip, rr);
                    sl.pi[p] = i;
                    sl.pj[p] = j;
                    st3(sl.v, N, i, vi);
                    st3(sl.v, N, j, vj);
                    p = (p + 1 < lead) ? p + 1 : (p < lead ? lead + (int)threadIdx.x : p + kThreads);
                }
                __syncthreads();
            }
            for (int i = threadIdx.x; i < n; i += kThreads) {
                double x[3];
                ld3(sl.v, N, i, x);
                st3(sl.vp, N, i, x);
            }
            __syncthreads();
            // ---- forward: moment correction
            if (A.correct) {
                const double ms[2] = {A.m[ic.a], A.m[ic.b]};
                {
                    Acc<double> acc[8];
                    for (int k = 0; k < 8; ++k) acc[k] = Acc<double>::zero();
                    for (int side = 0; side < nside; ++side) {
                        const int s0 = side ? b0 : a0, ns = side ? nb : na;
                        for (int q = threadIdx.x; q < ns; q += kThreads) {
                            const int i = s0 + q;
                            const double w = wg[cs + i], mp = ms[side] * w;
                            for (int k = 0; k < 3; ++k) acc[k].add(mp * (sl.v[k * N + i] - sl.vb[k * N + i]));
                            acc[3].add(mp * w);
                            acc[4 + side].add(w);
                        }
                    }
                    block_sum<double, 8>(acc, accp(sh.red_raw), accp(sh.red));
                    if (threadIdx.x == 0) {
                        const Acc<double>* r = accp(sh.red);
                        sh.Sw = r[3].x;
                        for (int k = 0; k < 3; ++k) {
                            sh.S[k] = r[k].x;
                            sh.B[k] = r[k].x / r[3].x;
                        }
                        sh.W1[0] = r[4].x;
                        sh.W1[1] = r[5].x;
                    }
                    __syncthreads();
                }
                {
                    Acc<double> acc[4];
                    for (int k = 0; k < 4; ++k) acc[k] = Acc<double>::zero();
                    for (int side = 0; side < nside; ++side) {
                        const int s0 = side ? b0 : a0, ns = side ? nb : na;
                        for (int q = threadIdx.x; q < ns; q += kThreads) {
                            const int i = s0 + q;
                            const double w = wg[cs + i], mp = ms[side] * w;
                            double dd = 0.0, v2 = 0.0;
                            for (int k = 0; k < 3; ++k) {
                                const double x = sl.v[k * N + i] - sh.B[k] * w, y = sl.vb[k * N + i];
                                sl.v[k * N + i] = x;
                                sl.vm[k * N + i] = x;
                                dd += (x - y) * (x + y);
                                v2 += x * x;
                            }
                            acc[0].add(0.5 * mp * dd);
                            acc[1 + side].add(0.5 * mp * v2);
                        }
                    }
                    block_sum<double, 4>(acc, accp(sh.red_raw), accp(sh.red));
                    if (threadIdx.x == 0) {
                        const Acc<double>* r = accp(sh.red);
                        const double dE = r[0].x;
                        sh.dE = dE;
                        sh.Es[0] = r[1].x;
                        sh.Es[1] = r[2].x;
                        double D0 = dE, D1 = 0.0;
                        int fail = 0;
                        if (!intra) {
                            const bool c0 = na >= 2, c1 = nb >= 2;
                            if (c0 && c1) {
                                const double wa = sh.W1[0] / (double)na * sh.Es[0];
                                const double wb = sh.W1[1] / (double)nb * sh.Es[1];
                                const double den = wa + wb;
                                if (den > 0.0) {
                                    D0 = wa / den * dE;
                                    D1 = dE - D0;
                                } else if (dE != 0.0) {
                                    fail = 1;
                                }
                            } else if (c0) {
                                D0 = dE;
                            } else if (c1) {
                                D0 = 0.0;
                                D1 = dE;
                            } else if (dE != 0.0) {
                                fail = 1;
                            }
                        }
                        sh.zeroed[0] = fabs(D0) <= 0x1p-47 * sh.Es[0];
                        sh.zeroed[1] = fabs(D1) <= 0x1p-47 * (intra ? 0.0 : sh.Es[1]);
                        sh.D[0] = sh.zeroed[0] ? 0.0 : D0;
                        sh.D[1] = sh.zeroed[1] ? 0.0 : D1;
                        sh.fail = fail;
                    }
                    __syncthreads();
                }
                // energy-pair order of each side: the permutation, stably sorted by descending weight (optional)
                for (int side = 0; side < nside; ++side) {
                    const int s0 = side ? b0 : a0, ns = side ? nb : na;
                    if (A.sort_by_weight) {
                        for (int r = threadIdx.x; r < ns; r += kThreads)
                            sl.keys[s0 + r] = weight_key(wg[cs + sl.perm[s0 + r]], (uint32_t)r);
                        __syncthreads();
                        block_sort_u64(sl.keys + s0, ns);
                        for (int r = threadIdx.x; r < ns; r += kThreads)
                            sl.rho[s0 + r] = sl.perm[s0 + (int)(sl.keys[s0 + r] & kPermMask)];
                    } else {
                        for (int r = threadIdx.x; r < ns; r += kThreads) sl.rho[s0 + r] = sl.perm[s0 + r];
                    }
                    __syncthreads();
                }
                // energy loops, in order, by one thread (the tape records every pair that absorbed energy)
                if (threadIdx.x == 0) {
                    int e = 0;
                    for (int side = 0; side < nside; ++side) {
                        sh.e0[side] = e;
                        sh.ne[side] = 0;
                        if (sh.fail) continue;
                        const int s0 = side ? b0 : a0, ns = side ? nb : na;
                        const double msd = ms[side];
                        if (sh.D[side] == 0.0) {
                            // Delta E_s vanishes here (exactly, or as rounding noise), so the step applies no energy
                            // pair; but it moves at first order with v and w, and then the first pair of the order
                            // absorbs it as the crossing pair. Tape that pair with U = 0 (no change in the forward).
                            for (int t = 0; t + 1 < ns; t += 2) {
                                const int i = sl.rho[s0 + t], j = sl.rho[s0 + t + 1];
                                double v1[3], v2[3];
                                ld3(sl.v, N, i, v1);
                                ld3(sl.v, N, j, v2);
                                const double K =
                                    pair_kecm<double, false>(A.c, msd * wg[cs + i], msd * wg[cs + j], v1, v2);
                                if (!(K > 0.0)) continue;
                                if (e < sl.E) {
                                    for (int k = 0; k < 3; ++k) {
                                        sl.ev[k * sl.E + e] = v1[k];
                                        sl.ev[(3 + k) * sl.E + e] = v2[k];
                                    }
                                    sl.ei[e] = i;
                                    sl.ej[e] = j;
                                    sl.eU[e] = 0.0;
                                    sl.eK[e] = K;
                                    sl.ecap[e] = 0;
                                    ++e;
                                    ++sh.ne[side];
                                }
                                break;
                            }
                            continue;
                        }
                        double D = sh.D[side];
                        for (int pass = 0; pass < A.max_corr_passes && D != 0.0; ++pass) {
                            for (int t = pass & 1; t + 1 < ns && D != 0.0; t += 2) {
                                const int i = sl.rho[s0 + t], j = sl.rho[s0 + t + 1];
                                double v1[3], v2[3];
                                ld3(sl.v, N, i, v1);
                                ld3(sl.v, N, j, v2);
                                const double m1 = msd * wg[cs + i], m2 = msd * wg[cs + j];
                                const double K = pair_kecm<double, false>(A.c, m1, m2, v1, v2);
                                if (!(K > 0.0)) continue;
                                const double capE = A.fE * K;
                                const double U = (D > 0.0 ? 1.0 : -1.0) * (fabs(D) < capE ? fabs(D) : capE);
                                if (e < sl.E) {
                                    for (int k = 0; k < 3; ++k) {
                                        sl.ev[k * sl.E + e] = v1[k];
                                        sl.ev[(3 + k) * sl.E + e] = v2[k];
                                    }
                                    sl.ei[e] = i;
                                    sl.ej[e] = j;
                                    sl.eU[e] = U;
                                    sl.eK[e] = K;
                                    sl.ecap[e] = !(fabs(D) < capE);
                                } else {
                                    latch(A.status, kErrTooLarge);
                                }
                                ++e;
                                ++sh.ne[side];
                                energy_pair<double, false>(A.c, m1, m2, K, v1, v2, U);
                                st3(sl.v, N, i, v1);
                                st3(sl.v, N, j, v2);
                                D -= U;
                            }
                        }
                        if (D != 0.0) sh.fail = 1;
                    }
                }
                __syncthreads();
                if (sh.fail && A.fail_policy == 0) {
                    for (int side = 0; side < nside; ++side) {
                        const int s0 = side ? b0 : a0, ns = side ? nb : na;
                        for (int q = threadIdx.x; q < ns; q += kThreads) {
                            double x[3];
                            ld3(sl.vb, N, s0 + q, x);
                            st3(sl.v, N, s0 + q, x);
                        }
                    }
                }
                if (sh.fail && A.fail_policy == 2 && threadIdx.x == 0) latch(A.status, kErrCorrectionFailed);
                __syncthreads();
            }
            if (G.tape == 1 && threadIdx.x == 0) {  // record: keep the per-cell scalars with the tape
                TapeHead& h = *sl.head;
                h.fail = A.correct ? sh.fail : 0;
                for (int k = 0; k < 2; ++k) {
                    h.ne[k] = sh.ne[k];
                    h.e0[k] = sh.e0[k];
                    h.zeroed[k] = sh.zeroed[k];
                    h.Es[k] = sh.Es[k];
                    h.W1[k] = sh.W1[k];
                    h.D[k] = sh.D[k];
                }
                for (int k = 0; k < 3; ++k) {
                    h.B[k] = sh.B[k];
                    h.S[k] = sh.S[k];
                }
                h.Sw = sh.Sw;
                h.dE = sh.dE;
            }
        }
        // ---- forward output
        if (G.ox) {
            for (int i = threadIdx.x; i < n; i += kThreads) {
                G.ox[cs + i] = sl.v[i];
                G.oy[cs + i] = sl.v[N + i];
                G.oz[cs + i] = sl.v[2 * N + i];
            }
        }
        // ---- reverse
        if (G.gx && active && !(A.correct && sh.fail && A.fail_policy == 0)) {
            for (int i = threadIdx.x; i < n; i += kThreads) {
                const double x[3] = {G.gx[cs + i], G.gy[cs + i], G.gz[cs + i]};
                st3(sl.g, N, i, x);
                const double z[3] = {0.0, 0.0, 0.0};
                st3(sl.gb, N, i, z);
            }
            __syncthreads();
            if (A.correct) {
                const double ms[2] = {A.m[ic.a], A.m[ic.b]};
                // energy pairs backwards (one thread; each side's pairs in reverse order)
                if (threadIdx.x == 0) {
                    for (int side = nside - 1; side >= 0; --side) {
                        sh.gD[side] = 0.0;
                        const int cnt = sh.ne[side] < sl.E - sh.e0[side] ? sh.ne[side] : sl.E - sh.e0[side];
                        if (cnt <= 0) continue;
                        const double msd = ms[side];
                        const double sgn = sh.D[side] > 0.0 ? 1.0 : -1.0;
                        double gUc = 0.0;
                        for (int k = sh.e0[side] + cnt - 1; k >= sh.e0[side]; --k) {
                            const int i = sl.ei[k], j = sl.ej[k];
                            double v1[3], v2[3], g1[3], g2[3], vr[3];
                            for (int d = 0; d < 3; ++d) {
                                v1[d] = sl.ev[d * sl.E + k];
                                v2[d] = sl.ev[(3 + d) * sl.E + k];
                                vr[d] = v1[d] - v2[d];
                            }
                            ld3(sl.g, N, i, g1);
                            ld3(sl.g, N, j, g2);
                            const double m1 = msd * wg[cs + i], m2 = msd * wg[cs + j], M = m1 + m2;
                            const double c1 = m2 / M, c2 = m1 / M, mu = m1 * m2 / M;
                            const double U = sl.eU[k], K = sl.eK[k];
                            const double x = U / K, gg = sqrt(1.0 - x), gm1 = -x / (1.0 + gg);
                            double h[3], ggm1 = 0.0, g1vr = 0.0, g2vr = 0.0, vr2 = 0.0;
                            for (int d = 0; d < 3; ++d) {
                                h[d] = c1 * g1[d] - c2 * g2[d];
                                ggm1 += h[d] * vr[d];
                                g1vr += g1[d] * vr[d];
                                g2vr += g2[d] * vr[d];
                                vr2 += vr[d] * vr[d];
                            }
                            double gvr[3] = {gm1 * h[0], gm1 * h[1], gm1 * h[2]};
                            const double gc1 = gm1 * g1vr, gc2 = -gm1 * g2vr;
                            double gK;
                            if (!sl.ecap[k]) {
                                // crossing pair: U = D - (earlier U); g - 1 depends on U and K
                                const double gU = -ggm1 / (2.0 * gg * K);
                                gK = ggm1 * x / (2.0 * gg * K);
                                gUc = gU;
                                sh.gD[side] += gU;
                            } else {
                                // capped pair: U = sign(D) fE K, so U/K is fixed; K still feeds the crossing U
                                gK = -gUc * sgn * A.fE;
                            }
                            for (int d = 0; d < 3; ++d) gvr[d] += gK * mu * vr[d];
                            const double gmu = gK * 0.5 * vr2;
                            const double M2 = M * M;
                            const double gm1m = gmu * m2 * m2 / M2 - gc1 * m2 / M2 + gc2 * m2 / M2;
                            const double gm2m = gmu * m1 * m1 / M2 + gc1 * m1 / M2 - gc2 * m1 / M2;
                            sl.gwl[i] += msd * gm1m;
                            sl.gwl[j] += msd * gm2m;
                            for (int d = 0; d < 3; ++d) {
                                g1[d] += gvr[d];
                                g2[d] -= gvr[d];
                            }
                            st3(sl.g, N, i, g1);
                            st3(sl.g, N, j, g2);
                        }
                    }
                    // Delta E split backwards
                    double gdE = 0.0, gE0 = 0.0, gE1 = 0.0, gW0 = 0.0, gW1 = 0.0;
                    const double g0 = sh.gD[0];
                    const double g1 = intra ? 0.0 : sh.gD[1];
                    if (intra) {
                        gdE = g0;
                    } else {
                        const bool c0 = na >= 2, c1 = nb >= 2;
                        if (c0 && c1) {
                            const double wa = sh.W1[0] / (double)na * sh.Es[0];
                            const double wb = sh.W1[1] / (double)nb * sh.Es[1];
                            const double den = wa + wb;
                            if (den > 0.0) {
                                const double f = wa / den;
                                gdE = g1 + (g0 - g1) * f;
                                const double gf = (g0 - g1) * sh.dE;
                                const double gwa = gf * wb / (den * den), gwb = -gf * wa / (den * den);
                                gW0 = gwa * sh.Es[0] / (double)na;
                                gE0 = gwa * sh.W1[0] / (double)na;
                                gW1 = gwb * sh.Es[1] / (double)nb;
                                gE1 = gwb * sh.W1[1] / (double)nb;
                            }
                        } else if (c0) {
                            gdE = g0;
                        } else if (c1) {
                            gdE = g1;
                        }
                    }
                    sh.gdE = gdE;
                    sh.gEs[0] = gE0;
                    sh.gEs[1] = gE1;
                    sh.gW1[0] = gW0;
                    sh.gW1[1] = gW1;
                }
                __syncthreads();
                // energy sums and the momentum shift backwards: g at v_pm, then g_B = -sum w g_vpm
                {
                    Acc<double> acc[3];
                    for (int k = 0; k < 3; ++k) acc[k] = Acc<double>::zero();
                    for (int side = 0; side < nside; ++side) {
                        const int s0 = side ? b0 : a0, ns = side ? nb : na;
                        const double msd = ms[side];
                        for (int q = threadIdx.x; q < ns; q += kThreads) {
                            const int i = s0 + q;
                            const double w = wg[cs + i], mp = msd * w;
                            double gm[3], xm[3], xb[3];
                            ld3(sl.g, N, i, gm);
                            ld3(sl.vm, N, i, xm);
                            ld3(sl.vb, N, i, xb);
                            const double gE = sh.gEs[side];
                            double xm2 = 0.0, xb2 = 0.0, gwd = 0.0;
                            for (int d = 0; d < 3; ++d) {
                                gm[d] += (sh.gdE + gE) * mp * xm[d];
                                sl.gb[d * N + i] -= sh.gdE * mp * xb[d];
                                xm2 += xm[d] * xm[d];
                                xb2 += xb[d] * xb[d];
                            }
                            gwd += sh.gdE * 0.5 * msd * (xm2 - xb2) + gE * 0.5 * msd * xm2 + sh.gW1[side];
                            for (int d = 0; d < 3; ++d) {
                                acc[d].add(-w * gm[d]);
                                gwd -= sh.B[d] * gm[d];
                            }
                            sl.gwl[i] += gwd;
                            st3(sl.g, N, i, gm);
                        }
                    }
                    block_sum<double, 3>(acc, accp(sh.red_raw), accp(sh.red));
                    if (threadIdx.x == 0) {
                        const Acc<double>* r = accp(sh.red);
                        double gSw = 0.0;
                        for (int d = 0; d < 3; ++d) {
                            sh.gS[d] = r[d].x / sh.Sw;
                            gSw -= r[d].x * sh.B[d] / sh.Sw;
                        }
                        sh.gSw = gSw;
                    }
                    __syncthreads();
                }
                // B = S / Sw, S = sum m w (v_ps - v_bs), Sw = sum m w^2 backwards
                for (int side = 0; side < nside; ++side) {
                    const int s0 = side ? b0 : a0, ns = side ? nb : na;
                    const double msd = ms[side];
                    for (int q = threadIdx.x; q < ns; q += kThreads) {
                        const int i = s0 + q;
                        const double w = wg[cs + i], mp = msd * w;
                        double gwd = 2.0 * mp * sh.gSw;
                        for (int d = 0; d < 3; ++d) {
                            sl.g[d * N + i] += mp * sh.gS[d];
                            sl.gb[d * N + i] -= mp * sh.gS[d];
                            gwd += msd * (sl.vp[d * N + i] - sl.vb[d * N + i]) * sh.gS[d];
                        }
                        sl.gwl[i] += gwd;
                    }
                }
                __syncthreads();
            }
            // scatter pairs backwards: rounds in reverse, the odd triplet in reverse by thread 0
            double glnl = 0.0;
            {
                const int npairs = intra ? ((na & 1) ? (na + 3) / 2 : na / 2) : (na > nb ? na : nb);
                const int nmin = intra ? na - 1 : (na < nb ? na : nb);
                const int lead = (intra && (na & 1)) ? 3 : 0;
                const int round = intra ? npairs : nmin;
                const int nround = (npairs + round - 1) / round;
                for (int rr = nround - 1; rr >= 0; --rr) {
                    const int r0 = rr * round;
                    const int r1 = r0 + round < npairs ? r0 + round : npairs;
                    // the triplet (0, 1, 2) shares particles: thread 0 undoes it in reverse; the other pairs of the round
                    // are disjoint from it and from each other
                    auto undo = [&](int p) {
                        const int i = sl.pi[p], j = sl.pj[p];
                        double vi[3], vj[3], g1[3], g2[3];
                        for (int k = 0; k < 3; ++k) {
                            vi[k] = sl.pv[k * N + p];
                            vj[k] = sl.pv[(3 + k) * N + p];
                        }
                        ld3(sl.g, N, i, g1);
                        ld3(sl.g, N, j, g2);
                        const uint4 r = draw(A.rng, (uint32_t)p, (uint32_t)c, ictr, kTagScat);
                        double gwi = 0.0, gwj = 0.0;
                        pair_reverse(A, ic, G.lnL, vi, vj, wg[cs + i], wg[cs + j], nmin, sl.pf[p], r, g1, g2, gwi, gwj,
                                     glnl);
                        st3(sl.g, N, i, g1);
                        st3(sl.g, N, j, g2);
                        sl.gwl[i] += gwi;
                        sl.gwl[j] += gwj;
                    };
                    if (lead && threadIdx.x == 0)
                        for (int p = lead - 1; p >= 0; --p) undo(p);
                    for (int p = r0 + lead + (int)threadIdx.x; p < r1; p += kThreads) undo(p);
                    __syncthreads();
                }
            }
            // dL/dv_before = scatter path + direct correction path; dL/dw, dL/dlnL accumulated
            for (int side = 0; side < nside; ++side) {
                const int s0 = side ? b0 : a0, ns = side ? nb : na;
                for (int q = threadIdx.x; q < ns; q += kThreads) {
                    const int i = s0 + q;
                    G.gx[cs + i] = sl.g[i] + sl.gb[i];
                    G.gy[cs + i] = sl.g[N + i] + sl.gb[N + i];
                    G.gz[cs + i] = sl.g[2 * N + i] + sl.gb[2 * N + i];
                    if (G.gw) G.gw[cs + i] += sl.gwl[i];
                }
            }
            {
                Acc<double> acc[1] = {Acc<double>{glnl}};
                block_sum<double, 1>(acc, accp(sh.red_raw), accp(sh.red));
                if (threadIdx.x == 0 && G.glnL) atomicAdd(G.glnL, accp(sh.red)[0].x);
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t adjoint_slab_bytes(int32_t max_cell, int32_t max_epairs) { return (slab_bytes(max_cell, max_epairs) + 255) & ~(size_t)255; }

cudaError_t launch_adjoint(const StepArgs& a, double lnL, double* ox, double* oy, double* oz, double* gx, double* gy,
                           double* gz, double* gw, double* glnL, char* slab, int32_t max_cell, int32_t max_epairs,
                           int32_t tape, int grid, cudaStream_t st)
{
    AdjArgs g;
    g.a = a;
    g.lnL = lnL;
    g.ox = ox;
    g.oy = oy;
    g.oz = oz;
    g.gx = gx;
    g.gy = gy;
    g.gz = gz;
    g.gw = gw;
    g.glnL = glnL;
    g.slab = slab;
    g.slab_stride = (int64_t)adjoint_slab_bytes(max_cell, max_epairs);
    g.max_cell = max_cell;
    g.max_epairs = max_epairs;
    g.tape = tape;
    k_adjoint<<<grid, kThreads, 0, st>>>(g);
    return cudaGetLastError();
}

}  // namespace mcc
