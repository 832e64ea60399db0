/*
 * moq_oracle.c -- the CPU oracle for multi-objective MaxCut sampling by noise-injected
 * simulated bifurcation (NI-SB), "Multi-Objective Optimization by Quantum-Annealing-
 * Inspired Algorithms" (arXiv 2604.26477).
 *
 * TEST INFRASTRUCTURE ONLY. Plain, slow, obviously-correct code: double precision for
 * the dynamics, int64 for cut values, __int128 for hypervolumes. It shares no code,
 * header or table with the CUDA library and is called only by the tests, the smoke
 * check and the CPU-baseline leg of the benchmark. Each function names the passage of
 * the paper it restates. Where the paper is silent or ambiguous the reading taken is
 * stated beside the code (the list of readings is kept with the design notes).
 *
 * Parity status of each function (what pins it, all in tests/):
 *   or_philox4x32_10  pinned: published known-answer vectors of Philox4x32-10.
 *   or_cuts           pinned: brute-force identities, hand-computed golden cuts.
 *   or_brute_force    pinned: enumeration identities (sum over all s, symmetry).
 *   or_pareto_filter  pinned: definition-based all-pairs check, hand golden fronts.
 *   or_hypervolume    pinned: the Appendix A worked example, inclusion-exclusion.
 *   or_das_dennis     pinned: lattice counts 190 (K=3) and 220 (K=4), binomial counts.
 *   or_sb             pinned: hand-computed steps, J=0 closed form, symmetry, max-cut
 *                     on bipartite graphs; trajectories are chaotic, so beyond a few
 *                     steps parity is statistical only.
 *   or_normal         pinned: moments, KS tests, the tail mass beyond 3 and 4.71 standard
 *                     deviations, no repeated values in 10^6 draws (53-bit uniforms); not
 *                     pinned bitwise (it goes through libm log/cos).
 *   or_dirichlet      pinned: simplex sums, moments of Dirichlet(1,..,1).
 *   or_mlp_*          pinned: central finite differences of the loss.
 *   or_e4m3           pinned: torch's float8_e4m3fn conversion (nearest even) on every
 *                     midpoint and random values, hand values (ties, saturation).
 *   or_force_e4m3     pinned: equals the one-step force of or_sb when every weight is
 *                     exact in E4M3; the row scales by hand; error bound 2^-4.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

/* ------------------------------------------------------------------------------------
 * Counter-based RNG: Philox4x32 with 10 rounds, from Salmon, Moraes, Dror and Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3" (SC'11), Sec. 3.3 / Table 2: each
 * round multiplies counter words 0 and 2 by two fixed odd constants, XORs the high
 * halves of the products with the other counter words and the key, and swaps; the
 * key is advanced by the two Weyl constants between rounds.
 * ---------------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout:
 *   initial state of spin i, replica r:  ctr = (0xFFFFFFFF, i, r, round), key = seed
 *     (the same definition as the CUDA sampler's, so both start from the same state);
 *   noise of spin i, replica r, step m:  ctr = (m, i, r, round), key = seed, one block
 *     per draw (the oracle's own stream: trajectories with noise are compared with the
 *     CUDA sampler's by distribution only). */
static void philox_at(uint64_t seed, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, uint32_t out[4])
{
    uint32_t ctr[4] = {w0, w1, w2, w3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

/* Gaussian eta_{i,m} of Eq. (NI-SB), a standard normal draw: Box-Muller (Box and Muller,
 * 1958) on two uniforms of full double resolution from the block at (m, i, r, round),
 *   u1 = (a + 1) 2^-53 in (0, 1],  a = the top 53 bits of words 0, 1 (o0 * 2^21 + o1 >> 11),
 *   u2 = b 2^-53 in [0, 1),        b = the same of words 2, 3,
 *   eta = sqrt(-2 ln u1) cos(2 pi u2).
 * The smallest u1 is 2^-53, so |eta| reaches 8.57: the tails are those of a Gaussian
 * to well below the probabilities any test here can see. */
double or_normal(uint64_t seed, uint64_t round, uint32_t r, uint32_t i, uint64_t m)
{
    uint32_t o[4];
    philox_at(seed, (uint32_t)m, i, r, (uint32_t)round, o);
    uint64_t a = ((uint64_t)o[0] << 21) | (o[1] >> 11);
    uint64_t b = ((uint64_t)o[2] << 21) | (o[3] >> 11);
    double u1 = ((double)a + 1.0) * 0x1p-53;
    double u2 = (double)b * 0x1p-53;
    double rho = sqrt(-2.0 * log(u1));
    return rho * cos(2.0 * M_PI * u2);
}

/* count consecutive steps m0, m0 + 1, .. of spin i, replica r (bulk draws for the tests) */
void or_normal_fill(uint64_t seed, uint64_t round, uint32_t r, uint32_t i, uint64_t m0, int64_t count, double* out)
{
    for (int64_t t = 0; t < count; ++t) out[t] = or_normal(seed, round, r, i, m0 + (uint64_t)t);
}

/* Uniform initial value in [-amp, amp): v = (w >> 8 - 2^23) * 2^-23 is exact in
 * float; amp * v is one IEEE single-precision product, so the CUDA sampler (which
 * forms the same product in float) starts from bitwise the same state. */
static double init_value(uint32_t word, float amp)
{
    float v = (float)((int32_t)(word >> 8) - 8388608) * 0x1p-23f;
    volatile float x = amp * v;
    return (double)x;
}

void or_initial_state(uint64_t seed, uint64_t round, uint32_t r, uint32_t i, float amp, double* x0, double* y0)
{
    uint32_t o[4];
    philox_at(seed, 0xFFFFFFFFu, i, r, (uint32_t)round, o);
    *x0 = init_value(o[0], amp);
    *y0 = init_value(o[1], amp);
}

/* ------------------------------------------------------------------------------------
 * Cut values, Eq. (single_obj): C_k(s) = 1/2 sum_{(i,j) in E} J^(k)_ij (1 - s_i s_j).
 * Spins are read from packed words: bit (i mod 64) of word i/64 is 1 when s_i = -1.
 * ---------------------------------------------------------------------------------- */
static int spin_of(const uint64_t* bits, int i)
{
    return ((bits[i >> 6] >> (i & 63)) & 1u) ? -1 : +1;
}

void or_cuts(int n, int K, int64_t E, const int32_t* ei, const int32_t* ej, const int32_t* w,
             int64_t M, const uint64_t* bits, int64_t* cuts /* M x K */)
{
    int W = (n + 63) / 64;
    for (int64_t s = 0; s < M; ++s) {
        const uint64_t* b = bits + s * W;
        for (int k = 0; k < K; ++k) {
            int64_t twice = 0;
            for (int64_t e = 0; e < E; ++e) {
                int si = spin_of(b, ei[e]), sj = spin_of(b, ej[e]);
                twice += (int64_t)w[(int64_t)k * E + e] * (int64_t)(1 - si * sj);
            }
            cuts[s * K + k] = twice / 2; /* (1 - s_i s_j) is 0 or 2: the sum is even */
        }
    }
}

/* Ising energies H_k(s) = sum_E J^(k)_ij s_i s_j ("Hamiltonian formulation"). */
void or_energies(int n, int K, int64_t E, const int32_t* ei, const int32_t* ej, const int32_t* w,
                 int64_t M, const uint64_t* bits, int64_t* H /* M x K */)
{
    int W = (n + 63) / 64;
    for (int64_t s = 0; s < M; ++s)
        for (int k = 0; k < K; ++k) {
            int64_t acc = 0;
            for (int64_t e = 0; e < E; ++e)
                acc += (int64_t)w[(int64_t)k * E + e] * spin_of(bits + s * W, ei[e]) * spin_of(bits + s * W, ej[e]);
            H[s * K + k] = acc;
        }
}

/* Brute force over the configuration space S = {-1,1}^n ("Hamiltonian formulation",
 * definition of P*): enumerate the 2^(n-1) configurations with s_0 = +1 (C(s) = C(-s),
 * so the other half repeats them). Configuration number c sets s_i = -1 for i >= 1
 * exactly when bit (i-1) of c is 1. Writes packed bits and cut vectors. */
void or_brute_force(int n, int K, int64_t E, const int32_t* ei, const int32_t* ej, const int32_t* w,
                    uint64_t* bits /* 2^(n-1) x W */, int64_t* cuts /* 2^(n-1) x K */)
{
    int W = (n + 63) / 64;
    int64_t count = (int64_t)1 << (n - 1);
    for (int64_t c = 0; c < count; ++c) {
        uint64_t* b = bits + c * W;
        memset(b, 0, sizeof(uint64_t) * W);
        for (int i = 1; i < n; ++i)
            if ((c >> (i - 1)) & 1)
                b[i >> 6] |= (uint64_t)1 << (i & 63);
        or_cuts(n, K, E, ei, ej, w, 1, b, cuts + c * K);
    }
}

/* ------------------------------------------------------------------------------------
 * Pareto dominance in cut-maximisation space ("Pareto filtering" section; the order of
 * the "Hamiltonian formulation" section written for C = maximised cuts instead of H):
 * u dominates v iff u_k >= v_k for every k and u_j > v_j for some j.
 * ---------------------------------------------------------------------------------- */
int or_dominates(int K, const int64_t* u, const int64_t* v)
{
    int strictly = 0;
    for (int k = 0; k < K; ++k) {
        if (u[k] < v[k]) return 0;
        if (u[k] > v[k]) strictly = 1;
    }
    return strictly;
}

static int weakly_dominates(int K, const int64_t* u, const int64_t* v)
{
    for (int k = 0; k < K; ++k)
        if (u[k] < v[k]) return 0;
    return 1;
}

/* Pareto filter with deduplication of objective vectors ("Pareto filtering"): keep the
 * distinct cut vectors of the pool that no pool member dominates; each kept vector is
 * represented by its lowest pool index. Plain insertion into an archive, in pool order:
 * a candidate equal to or dominated by a member is dropped; otherwise the members it
 * dominates leave and it enters. Returns the archive size; keep[] holds pool indices in
 * ascending order. */
int64_t or_pareto_filter(int K, int64_t M, const int64_t* cuts, int64_t* keep)
{
    int64_t F = 0;
    for (int64_t c = 0; c < M; ++c) {
        const int64_t* u = cuts + c * K;
        int covered = 0;
        for (int64_t a = 0; a < F && !covered; ++a)
            covered = weakly_dominates(K, cuts + keep[a] * K, u);
        if (covered) continue;
        int64_t out = 0;
        for (int64_t a = 0; a < F; ++a)
            if (!or_dominates(K, u, cuts + keep[a] * K))
                keep[out++] = keep[a];
        keep[out++] = c;
        F = out;
    }
    return F;
}

/* ------------------------------------------------------------------------------------
 * Hypervolume ("Hamiltonian formulation" Eq. HV and Appendix A): the Lebesgue measure
 * of the union of boxes prod_k [r_k, y_k] over the front. Computed exactly in integers
 * by slicing the last objective (While, Hingston, Barone, Huband, "A faster algorithm
 * for calculating hypervolume", IEEE TEVC 2006): sort by y_K descending; the slab
 * between consecutive y_K values is covered in the first K-1 objectives by exactly the
 * points above it, so HV_K = sum_t (y_K[t] - y_K[t+1]) * HV_{K-1}(first t+1 points),
 * with y_K[F] = r_K. In two objectives the slices are the staircase of Appendix A.
 * A point with some y_k < r_k spans an empty box and is left out.
 * ---------------------------------------------------------------------------------- */
static int g_sort_dim;
static const int64_t* g_sort_pts;
static int g_sort_stride;
static int cmp_desc(const void* a, const void* b)
{
    int64_t ia = *(const int64_t*)a, ib = *(const int64_t*)b;
    int64_t va = g_sort_pts[ia * g_sort_stride + g_sort_dim], vb = g_sort_pts[ib * g_sort_stride + g_sort_dim];
    if (va > vb) return -1;
    if (va < vb) return 1;
    return (ia > ib) - (ia < ib);
}

static void sort_desc(int64_t* idx, int64_t F, const int64_t* pts, int stride, int dim)
{
    g_sort_dim = dim;
    g_sort_pts = pts;
    g_sort_stride = stride;
    qsort(idx, (size_t)F, sizeof(int64_t), cmp_desc);
}

/* HV of points idx[0..F) in objectives 0..D-1 */
static i128 hv_slice(int D, int64_t F, const int64_t* idx, const int64_t* pts, int stride, const int64_t* ref)
{
    if (F == 0) return 0;
    int64_t* s = (int64_t*)malloc(sizeof(int64_t) * F);
    memcpy(s, idx, sizeof(int64_t) * F);
    sort_desc(s, F, pts, stride, D - 1);
    i128 vol = 0;
    if (D == 1) {
        vol = (i128)(pts[s[0] * stride] - ref[0]);
    } else if (D == 2) {
        /* staircase: widest first; each point adds the strip above the best y_2 so far */
        /* (sorted here by y_2 descending, so it is the mirror image: strips in y_1) */
        int64_t best1 = ref[0];
        for (int64_t t = 0; t < F; ++t) {
            const int64_t* p = pts + s[t] * stride;
            if (p[0] > best1) {
                vol += (i128)(p[0] - best1) * (i128)(p[1] - ref[1]);
                best1 = p[0];
            }
        }
    } else {
        for (int64_t t = 0; t < F; ++t) {
            int64_t top = pts[s[t] * stride + D - 1];
            int64_t below = (t + 1 < F) ? pts[s[t + 1] * stride + D - 1] : ref[D - 1];
            if (top > below)
                vol += (i128)(top - below) * hv_slice(D - 1, t + 1, s, pts, stride, ref);
        }
    }
    free(s);
    return vol;
}

/* out[0] = low 64 bits, out[1] = high 64 bits (two's complement of the __int128) */
void or_hypervolume(int K, int64_t F, const int64_t* pts /* F x K */, const int64_t* ref, int64_t out[2])
{
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (F > 0 ? F : 1));
    int64_t m = 0;
    for (int64_t p = 0; p < F; ++p) {
        int inside = 1;
        for (int k = 0; k < K; ++k)
            if (pts[p * K + k] < ref[k]) inside = 0;
        if (inside) idx[m++] = p;
    }
    i128 v = hv_slice(K, m, idx, pts, K, ref);
    free(idx);
    out[0] = (int64_t)(uint64_t)v;
    out[1] = (int64_t)(v >> 64);
}

/* ------------------------------------------------------------------------------------
 * Weight vectors ("Scalarization via the weighted sum method", Appendix B): the
 * Das-Dennis simplex lattice of resolution H, all c in {0, 1/H, ..., 1}^K with
 * sum c = 1; with interior != 0 only points with every c_k > 0 (the paper removes the
 * vertices and edges of the simplex). Order: lexicographically ascending (m_1..m_K).
 * Returns the count; writes c when out != NULL.
 * ---------------------------------------------------------------------------------- */
static int64_t dd_rec(int K, int H, int lo, int k, int left, int* m, double* out, int64_t cnt)
{
    if (k == K - 1) {
        if (left < lo) return cnt;
        m[k] = left;
        if (out)
            for (int q = 0; q < K; ++q) out[cnt * K + q] = (double)m[q] / (double)H;
        return cnt + 1;
    }
    for (int v = lo; v <= left; ++v) {
        m[k] = v;
        cnt = dd_rec(K, H, lo, k + 1, left - v, m, out, cnt);
    }
    return cnt;
}

int64_t or_das_dennis(int K, int H, int interior, double* out)
{
    int m[64];
    if (K < 1 || K > 64 || H < 1) return 0;
    return dd_rec(K, H, interior ? 1 : 0, 0, H, m, out, 0);
}

/* Uniform weight vectors on the simplex (Dirichlet(1,..,1), the alternative to the
 * lattice shown in Appendix B): c_k = e_k / sum_q e_q with e_k = -ln u_k, u_k uniform
 * in (0, 1] from Philox ctr = (r, k >> 2, 0x4C414D42, round), word k & 3. */
void or_dirichlet(int R, int K, uint64_t seed, uint64_t round, double* out /* R x K */)
{
    for (int r = 0; r < R; ++r) {
        double e[64], sum = 0.0;
        for (int k = 0; k < K; ++k) {
            uint32_t o[4];
            philox_at(seed, (uint32_t)r, (uint32_t)(k >> 2), 0x4C414D42u, (uint32_t)round, o);
            double u = ((double)(o[k & 3] >> 8) + 1.0) * 0x1p-24;
            e[k] = -log(u);
            sum += e[k];
        }
        for (int k = 0; k < K; ++k) out[(int64_t)r * K + k] = e[k] / sum;
    }
}

/* ------------------------------------------------------------------------------------
 * Noise-injected simulated bifurcation ("Simulated Bifurcation with Gaussian noise",
 * the SB equations and Eq. NI-SB), one replica per weight vector lambda_r:
 *
 *   J(c)_ij = sum_k c_k J^(k)_ij                     (Eq. H_total)
 *   c0      = 1 / max_i |sum_j J(c)_ij|
 *   dx_i/dt = a0 y_i
 *   dy_i/dt = -(a0 - a(t)) x_i + c0 sum_j Jt_ij phi(x_j) + alpha eta_i
 *   phi(x)  = x (bSB) or sgn(x) (dSB);  s_i = sgn(x_i) at the end
 *
 * Readings where the paper is silent or ambiguous:
 *  - Jt = -J(c): SB as printed climbs sum J phi phi, while H_total is minimised, so the
 *    dynamics run on the negated coupling (then maximal cuts are the attractors).
 *  - Integration: Euler with step dt in the symplectic order: y from the current x
 *    and phi(x), then x from the new y, then the inelastic wall (|x_i| > 1 ->
 *    x_i = sgn(x_i), y_i = 0).
 *  - Noise enters as y += dt * alpha * eta (noise_sqrt_dt = 0), the Euler step of the
 *    printed equation; noise_sqrt_dt = 1 gives the Euler-Maruyama alpha sqrt(dt) eta.
 *  - a(t): a_m = a0 m / (T - 1) for m = 0..T-1 (a_0 = 0 when T = 1), or a given array.
 *  - c0: if every row sum of J(c) vanishes, 1 / max_i sum_j |J(c)_ij|; if J(c) = 0, 1.
 *  - sgn(0) = +1, so spins are exactly +-1; the wall test is strict.
 *  - Initial x, y uniform in [-init_amp, init_amp) (see init_value).
 *
 * lambda: R x K doubles. x_init/y_init (R x n) override the Philox start when given.
 * Outputs: bits (R x W packed spins), optionally x_out, y_out (R x n) and c0_out (R).
 * ---------------------------------------------------------------------------------- */
int or_sb(int n, int K, int64_t E, const int32_t* ei, const int32_t* ej, const int32_t* w,
          int R, const double* lambda,
          int variant /* 0 = dSB, 1 = bSB */, int T, double dt, double a0, double alpha,
          float init_amp, const double* schedule, int noise_sqrt_dt,
          uint64_t seed, uint64_t round,
          const double* x_init, const double* y_init,
          uint64_t* bits, double* x_out, double* y_out, double* c0_out)
{
    int W = (n + 63) / 64;
    int64_t* rowsum = (int64_t*)calloc((size_t)n * K, sizeof(int64_t));
    for (int64_t e = 0; e < E; ++e)
        for (int k = 0; k < K; ++k) {
            rowsum[(int64_t)ei[e] * K + k] += w[(int64_t)k * E + e];
            rowsum[(int64_t)ej[e] * K + k] += w[(int64_t)k * E + e];
        }
    int status = 0;
#pragma omp parallel for schedule(dynamic, 4)
    for (int r = 0; r < R; ++r) {
        const double* c = lambda + (int64_t)r * K;
        double* x = (double*)malloc(sizeof(double) * n);
        double* y = (double*)malloc(sizeof(double) * n);
        double* f = (double*)malloc(sizeof(double) * n);
        double* phi = (double*)malloc(sizeof(double) * n);
        double* Jc = (double*)malloc(sizeof(double) * (E > 0 ? E : 1));
        double* absrow = (double*)calloc((size_t)n, sizeof(double));

        /* J(c) per edge, Eq. H_total */
        for (int64_t e = 0; e < E; ++e) {
            double v = 0.0;
            for (int k = 0; k < K; ++k) v += c[k] * (double)w[(int64_t)k * E + e];
            Jc[e] = v;
            absrow[ei[e]] += fabs(v);
            absrow[ej[e]] += fabs(v);
        }
        /* c0 = 1 / max_i |sum_j J(c)_ij|, from the integer row sums */
        double mx = 0.0, mxabs = 0.0;
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int k = 0; k < K; ++k) s += c[k] * (double)rowsum[(int64_t)i * K + k];
            if (fabs(s) > mx) mx = fabs(s);
            if (absrow[i] > mxabs) mxabs = absrow[i];
        }
        double c0 = mx > 0.0 ? 1.0 / mx : (mxabs > 0.0 ? 1.0 / mxabs : 1.0);
        if (c0_out) c0_out[r] = c0;

        for (int i = 0; i < n; ++i) {
            if (x_init) {
                x[i] = x_init[(int64_t)r * n + i];
                y[i] = y_init ? y_init[(int64_t)r * n + i] : 0.0;
            } else {
                or_initial_state(seed, round, (uint32_t)r, (uint32_t)i, init_amp, &x[i], &y[i]);
            }
        }
        for (int m = 0; m < T; ++m) {
            double a = schedule ? schedule[m] : (T > 1 ? a0 * (double)m / (double)(T - 1) : 0.0);
            for (int i = 0; i < n; ++i)
                phi[i] = (variant == 0) ? (x[i] >= 0.0 ? 1.0 : -1.0) : x[i];
            for (int i = 0; i < n; ++i) f[i] = 0.0;
            for (int64_t e = 0; e < E; ++e) { /* Jt = -J(c) */
                f[ei[e]] += -Jc[e] * phi[ej[e]];
                f[ej[e]] += -Jc[e] * phi[ei[e]];
            }
            for (int i = 0; i < n; ++i) {
                double drift = -(a0 - a) * x[i] + c0 * f[i];
                double noise = 0.0;
                if (alpha != 0.0)
                    noise = alpha * or_normal(seed, round, (uint32_t)r, (uint32_t)i, (uint64_t)m);
                if (noise_sqrt_dt)
                    y[i] = y[i] + dt * drift + sqrt(dt) * noise;
                else
                    y[i] = y[i] + dt * (drift + noise);
                x[i] = x[i] + dt * a0 * y[i];
                if (fabs(x[i]) > 1.0) {
                    x[i] = x[i] > 0.0 ? 1.0 : -1.0;
                    y[i] = 0.0;
                }
            }
        }
        uint64_t* b = bits + (int64_t)r * W;
        for (int q = 0; q < W; ++q) b[q] = 0;
        for (int i = 0; i < n; ++i) {
            if (x[i] < 0.0) b[i >> 6] |= (uint64_t)1 << (i & 63);
            if (x_out) x_out[(int64_t)r * n + i] = x[i];
            if (y_out) y_out[(int64_t)r * n + i] = y[i];
        }
        free(x); free(y); free(f); free(phi); free(Jc); free(absrow);
    }
    free(rowsum);
    return status;
}

/* ------------------------------------------------------------------------------------
 * FP8 operands of the dense dSB force (the precision growth of the force contraction;
 * the paper itself runs float16). E4M3 (the OCP 8-bit floating-point format): a sign,
 * 4 exponent bits with bias 7 and 3 mantissa bits; the normal values are
 * (1 + m/8) 2^(e-7) for e = 1..15 except e = 15, m = 7 (NaN), the subnormal ones m 2^-9,
 * so the largest finite value is 448. or_e4m3 returns the value of that set nearest to v,
 * on a tie the one whose mantissa field m is even, saturating at +-448; it walks the 127
 * non-negative values in increasing order, by the definition.
 * ---------------------------------------------------------------------------------- */
double or_e4m3(double v)
{
    double a = fabs(v), best = 0.0, bestd = a;
    int bestm = 0;
    for (int e = 0; e <= 15; ++e)
        for (int m = 0; m <= 7; ++m) {
            if (e == 15 && m == 7) continue;
            double val = (e == 0) ? ldexp((double)m, -9) : ldexp(1.0 + m / 8.0, e - 7);
            double d = fabs(a - val);
            if (d < bestd || (d == bestd && (m & 1) == 0 && (bestm & 1) == 1)) {
                best = val;
                bestd = d;
                bestm = m;
            }
        }
    if (a > 448.0) best = 448.0;
    return v < 0.0 ? -best : best;
}

/* The couplings the FP8 force uses (reading: one power-of-two scale per row and
 * objective). For row i of objective k, s = 2^e with e >= 0 the smallest exponent such
 * that max_j |J^(k)_ij| <= 448 s, and the coupling J^(k)_ij enters row i as
 * s * E4M3(J^(k)_ij / s). An edge e = (ei, ej) thus has one value for row ei (wq_i) and
 * one for row ej (wq_j), both K x E; scale is K x n. */
void or_e4m3_couplings(int n, int K, int64_t E, const int32_t* ei, const int32_t* ej, const int32_t* w,
                       double* wq_i, double* wq_j, double* scale)
{
    for (int k = 0; k < K; ++k) {
        double* sc = scale + (int64_t)k * n;
        double* mx = (double*)calloc((size_t)n, sizeof(double));
        for (int64_t e = 0; e < E; ++e) {
            double a = fabs((double)w[(int64_t)k * E + e]);
            if (a > mx[ei[e]]) mx[ei[e]] = a;
            if (a > mx[ej[e]]) mx[ej[e]] = a;
        }
        for (int i = 0; i < n; ++i) {
            double s = 1.0;
            while (mx[i] > 448.0 * s) s *= 2.0;
            sc[i] = s;
        }
        for (int64_t e = 0; e < E; ++e) {
            double v = (double)w[(int64_t)k * E + e];
            wq_i[(int64_t)k * E + e] = sc[ei[e]] * or_e4m3(v / sc[ei[e]]);
            wq_j[(int64_t)k * E + e] = sc[ej[e]] * or_e4m3(v / sc[ej[e]]);
        }
        free(mx);
    }
}

/* The SB force c0 sum_j (-J(c)_ij) phi_j (SB equations, negated coupling) of R replicas
 * with the couplings of or_e4m3_couplings: J(c)_ij = sum_k c_k wq^(k) of the edge as seen
 * from row i. c0 (R) is given (the FP8 step keeps the c0 of the exact weights). phi and
 * f are R x n. */
void or_force_e4m3(int n, int K, int64_t E, const int32_t* ei, const int32_t* ej, const double* wq_i, const double* wq_j,
                   int R, const double* lambda, const double* c0, const double* phi, double* f)
{
    for (int r = 0; r < R; ++r) {
        const double* c = lambda + (int64_t)r * K;
        const double* p = phi + (int64_t)r * n;
        double* fr = f + (int64_t)r * n;
        for (int i = 0; i < n; ++i) fr[i] = 0.0;
        for (int64_t e = 0; e < E; ++e) {
            double ji = 0.0, jj = 0.0;
            for (int k = 0; k < K; ++k) {
                ji += c[k] * wq_i[(int64_t)k * E + e];
                jj += c[k] * wq_j[(int64_t)k * E + e];
            }
            fr[ei[e]] += -ji * p[ej[e]];
            fr[ej[e]] += -jj * p[ei[e]];
        }
        for (int i = 0; i < n; ++i) fr[i] *= c0[r];
    }
}

/* Reference point r_k = sum_E min(0, J^(k)_e): every cut value satisfies C_k(s) >= r_k
 * (each edge adds J or 0), so r is dominated by every sample, as the HV definition
 * requires. */
void or_reference_point(int K, int64_t E, const int32_t* w, int64_t* ref)
{
    for (int k = 0; k < K; ++k) {
        int64_t s = 0;
        for (int64_t e = 0; e < E; ++e)
            if (w[(int64_t)k * E + e] < 0) s += w[(int64_t)k * E + e];
        ref[k] = s;
    }
}

/* ------------------------------------------------------------------------------------
 * Learned weight-vector proposal (not in the paper: the surrogate model of the learned
 * proposal). A multilayer perceptron maps an input row x (D_in values: the weight vector
 * and graph statistics) to D_out predictions:
 *   h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  y = W3 h2 + b3
 * with W1: H x D_in, W2: H x H, W3: D_out x H. Parameters are one flat vector in the order
 * W1, b1, W2, b2, W3, b3 (row-major). Loss over a batch of B rows with targets t:
 *   L = 1 / (B D_out) sum_b sum_k (y_bk - t_bk)^2.
 * or_mlp_forward writes y (B x D_out); or_mlp_loss_grad returns L and writes dL/dparams.
 * ---------------------------------------------------------------------------------- */
static void mlp_layer_offsets(int din, int h, int dout, int64_t off[6])
{
    off[0] = 0;                          /* W1 */
    off[1] = off[0] + (int64_t)h * din;  /* b1 */
    off[2] = off[1] + h;                 /* W2 */
    off[3] = off[2] + (int64_t)h * h;    /* b2 */
    off[4] = off[3] + h;                 /* W3 */
    off[5] = off[4] + (int64_t)dout * h; /* b3 */
}

int64_t or_mlp_param_count(int din, int h, int dout)
{
    int64_t off[6];
    mlp_layer_offsets(din, h, dout, off);
    return off[5] + dout;
}

static void mlp_forward_row(int din, int h, int dout, const double* p, const double* x, double* a1, double* h1,
                            double* a2, double* h2, double* y)
{
    int64_t off[6];
    mlp_layer_offsets(din, h, dout, off);
    for (int j = 0; j < h; ++j) {
        double s = p[off[1] + j];
        for (int i = 0; i < din; ++i) s += p[off[0] + (int64_t)j * din + i] * x[i];
        a1[j] = s;
        h1[j] = s > 0.0 ? s : 0.0;
    }
    for (int j = 0; j < h; ++j) {
        double s = p[off[3] + j];
        for (int i = 0; i < h; ++i) s += p[off[2] + (int64_t)j * h + i] * h1[i];
        a2[j] = s;
        h2[j] = s > 0.0 ? s : 0.0;
    }
    for (int k = 0; k < dout; ++k) {
        double s = p[off[5] + k];
        for (int i = 0; i < h; ++i) s += p[off[4] + (int64_t)k * h + i] * h2[i];
        y[k] = s;
    }
}

void or_mlp_forward(int din, int h, int dout, const double* p, int64_t B, const double* X, double* Y)
{
    double* buf = (double*)malloc(sizeof(double) * 4 * h);
    for (int64_t b = 0; b < B; ++b)
        mlp_forward_row(din, h, dout, p, X + b * din, buf, buf + h, buf + 2 * h, buf + 3 * h, Y + b * dout);
    free(buf);
}

/* Backpropagation written out per row: dy = 2 (y - t) / (B D_out); the gradient of each
 * layer is the outer product of the incoming gradient and the layer input; relu passes
 * the gradient where its pre-activation is positive. */
double or_mlp_loss_grad(int din, int h, int dout, const double* p, int64_t B, const double* X, const double* T, double* grad)
{
    int64_t off[6];
    mlp_layer_offsets(din, h, dout, off);
    const int64_t P = off[5] + dout;
    for (int64_t q = 0; q < P; ++q) grad[q] = 0.0;
    double* a1 = (double*)malloc(sizeof(double) * 7 * h + sizeof(double) * dout * 2);
    double *h1 = a1 + h, *a2 = h1 + h, *h2 = a2 + h, *d2 = h2 + h, *d1 = d2 + h, *tmp = d1 + h;
    double *y = tmp + h, *dy = y + dout;
    double loss = 0.0;
    const double scale = 1.0 / ((double)B * dout);
    for (int64_t b = 0; b < B; ++b) {
        const double* x = X + b * din;
        mlp_forward_row(din, h, dout, p, x, a1, h1, a2, h2, y);
        for (int k = 0; k < dout; ++k) {
            const double e = y[k] - T[b * dout + k];
            loss += e * e * scale;
            dy[k] = 2.0 * e * scale;
        }
        /* layer 3 */
        for (int k = 0; k < dout; ++k) {
            grad[off[5] + k] += dy[k];
            for (int i = 0; i < h; ++i) grad[off[4] + (int64_t)k * h + i] += dy[k] * h2[i];
        }
        for (int i = 0; i < h; ++i) {
            double s = 0.0;
            for (int k = 0; k < dout; ++k) s += p[off[4] + (int64_t)k * h + i] * dy[k];
            d2[i] = a2[i] > 0.0 ? s : 0.0;
        }
        /* layer 2 */
        for (int j = 0; j < h; ++j) {
            grad[off[3] + j] += d2[j];
            for (int i = 0; i < h; ++i) grad[off[2] + (int64_t)j * h + i] += d2[j] * h1[i];
        }
        for (int i = 0; i < h; ++i) {
            double s = 0.0;
            for (int j = 0; j < h; ++j) s += p[off[2] + (int64_t)j * h + i] * d2[j];
            d1[i] = a1[i] > 0.0 ? s : 0.0;
        }
        /* layer 1 */
        for (int j = 0; j < h; ++j) {
            grad[off[1] + j] += d1[j];
            for (int i = 0; i < din; ++i) grad[off[0] + (int64_t)j * din + i] += d1[j] * x[i];
        }
    }
    free(a1);
    return loss;
}

/* ------------------------------------------------------------------------------------
 * The same network with BF16 operands (the tensor-core surrogate's arithmetic; not in the
 * paper). rho(v) rounds v to the nearest BF16 value (8 significant bits, the FP32
 * exponent range, ties to an even significand; below 2^-126 multiples of 2^-133). Every
 * matrix-product operand is rounded, every sum and every bias gradient is exact:
 *   x~ = rho(x); a1 = W1 x~ + b1; h1~ = rho(relu(a1)); a2 = W2 h1~ + b2;
 *   h2~ = rho(relu(a2)); y = W3 h2~ + b3; dy = 2 (y - t) / (B D_out); dy~ = rho(dy);
 *   d2 = (W3^T dy~) [a2 > 0]; d2~ = rho(d2); d1 = (W2^T d2~) [a1 > 0]; d1~ = rho(d1);
 *   dW3 = sum dy~ h2~^T, db3 = sum dy; dW2 = sum d2~ h1~^T, db2 = sum d2;
 *   dW1 = sum d1~ x~^T, db1 = sum d1.
 * The weights are taken as given (the caller passes BF16 values).
 * ---------------------------------------------------------------------------------- */
double or_bf16(double v)
{
    if (v == 0.0 || isnan(v) || isinf(v)) return v;
    const double a = fabs(v);
    if (a < 0x1p-126) return nearbyint(v * 0x1p133) * 0x1p-133; /* subnormal BF16 spacing */
    int e;
    const double f = frexp(v, &e); /* v = f 2^e, 0.5 <= |f| < 1 */
    const double r = nearbyint(f * 256.0) * 0x1p-8; /* 8 significant bits, ties to even */
    const double out = ldexp(r, e);
    return fabs(out) > 0x1.FEp127 ? copysign(INFINITY, v) : out;
}

static void mlp_forward_row_bf16(int din, int h, int dout, const double* p, const double* x, double* xr, double* a1,
                                 double* h1, double* a2, double* h2, double* y)
{
    int64_t off[6];
    mlp_layer_offsets(din, h, dout, off);
    for (int i = 0; i < din; ++i) xr[i] = or_bf16(x[i]);
    for (int j = 0; j < h; ++j) {
        double s = p[off[1] + j];
        for (int i = 0; i < din; ++i) s += p[off[0] + (int64_t)j * din + i] * xr[i];
        a1[j] = s;
        h1[j] = or_bf16(s > 0.0 ? s : 0.0);
    }
    for (int j = 0; j < h; ++j) {
        double s = p[off[3] + j];
        for (int i = 0; i < h; ++i) s += p[off[2] + (int64_t)j * h + i] * h1[i];
        a2[j] = s;
        h2[j] = or_bf16(s > 0.0 ? s : 0.0);
    }
    for (int k = 0; k < dout; ++k) {
        double s = p[off[5] + k];
        for (int i = 0; i < h; ++i) s += p[off[4] + (int64_t)k * h + i] * h2[i];
        y[k] = s;
    }
}

void or_mlp_forward_bf16(int din, int h, int dout, const double* p, int64_t B, const double* X, double* Y)
{
    double* buf = (double*)malloc(sizeof(double) * (4 * h + din));
    for (int64_t b = 0; b < B; ++b)
        mlp_forward_row_bf16(din, h, dout, p, X + b * din, buf + 4 * h, buf, buf + h, buf + 2 * h, buf + 3 * h, Y + b * dout);
    free(buf);
}

double or_mlp_loss_grad_bf16(int din, int h, int dout, const double* p, int64_t B, const double* X, const double* T, double* grad)
{
    int64_t off[6];
    mlp_layer_offsets(din, h, dout, off);
    const int64_t P = off[5] + dout;
    for (int64_t q = 0; q < P; ++q) grad[q] = 0.0;
    double* a1 = (double*)malloc(sizeof(double) * (8 * h + 3 * dout + din));
    double *h1 = a1 + h, *a2 = h1 + h, *h2 = a2 + h, *d2 = h2 + h, *d1 = d2 + h, *d2r = d1 + h, *d1r = d2r + h;
    double *y = d1r + h, *dy = y + dout, *dyr = dy + dout, *xr = dyr + dout;
    double loss = 0.0;
    const double scale = 1.0 / ((double)B * dout);
    for (int64_t b = 0; b < B; ++b) {
        mlp_forward_row_bf16(din, h, dout, p, X + b * din, xr, a1, h1, a2, h2, y);
        for (int k = 0; k < dout; ++k) {
            const double e = y[k] - T[b * dout + k];
            loss += e * e * scale;
            dy[k] = 2.0 * e * scale;
            dyr[k] = or_bf16(dy[k]);
        }
        for (int k = 0; k < dout; ++k) {
            grad[off[5] + k] += dy[k];
            for (int i = 0; i < h; ++i) grad[off[4] + (int64_t)k * h + i] += dyr[k] * h2[i];
        }
        for (int i = 0; i < h; ++i) {
            double s = 0.0;
            for (int k = 0; k < dout; ++k) s += p[off[4] + (int64_t)k * h + i] * dyr[k];
            d2[i] = a2[i] > 0.0 ? s : 0.0;
            d2r[i] = or_bf16(d2[i]);
        }
        for (int j = 0; j < h; ++j) {
            grad[off[3] + j] += d2[j];
            for (int i = 0; i < h; ++i) grad[off[2] + (int64_t)j * h + i] += d2r[j] * h1[i];
        }
        for (int i = 0; i < h; ++i) {
            double s = 0.0;
            for (int j = 0; j < h; ++j) s += p[off[2] + (int64_t)j * h + i] * d2r[j];
            d1[i] = a1[i] > 0.0 ? s : 0.0;
            d1r[i] = or_bf16(d1[i]);
        }
        for (int j = 0; j < h; ++j) {
            grad[off[1] + j] += d1[j];
            for (int i = 0; i < din; ++i) grad[off[0] + (int64_t)j * din + i] += d1r[j] * xr[i];
        }
    }
    free(a1);
    return loss;
}
