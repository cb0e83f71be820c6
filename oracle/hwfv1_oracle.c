/*
 * hwfv1_oracle.c -- plain, slow CPU statement of the adaptive Haar-wavelet
 * first-order finite-volume shallow-water model (HWFV1) of Chowdhury,
 * Kesserwani, Rouge & Richmond, "GPU-parallelisation of wavelet-based grid
 * adaptation for fast finite volume modelling" (arXiv 2206.05761).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity oracle for the CUDA
 * library in paper_2206_05761_gb300/.  Only tests/, __graft_entry__.smoke()
 * and the cpu_baseline / --impl reference legs of bench.py may load it.  It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * Style: everything is written the obvious way, for a reader checking it
 * against the paper by eye.  Each grid level n is a row-major array of
 * 2^n x 2^n cells (index j*2^n + i, j grows with y), the hierarchy of all
 * levels is stored level after level (level n starts at (4^n-1)/3), leaves
 * are found by the recursive depth-first traversal of Algorithm 2, and the
 * FV1 update is one call per leaf.  Compile with -ffp-contract=off so that
 * no multiply-add is fused: the operation order written here is the
 * normative one.
 *
 * Readings of points where the paper is silent (each is also listed in the
 * design notes of the repository):
 *  R-taps   Eq. 3/4 filter taps (footnote 1 leaves them out): encode uses
 *           H0=H1=G0=1/2, G1=-1/2, decode H0=H1=G0=1, G1=-1, so that a
 *           parent coefficient is the average of its four children.  The
 *           exact power-of-two scalings are applied once, after the sums,
 *           in the bracketing of Eq. 3a-3d / 4a-4d.
 *  R-norm   normalised detail (Sec. 2.1.2) uses absolute values,
 *           max(|da|,|db|,|dg|), and s_max,q = max(1, max |s_q^(L)|) over the
 *           finest grid; the test is the division-free form
 *           max(|da|,|db|,|dg|) >= (eps * 2^(n-L)) * s_max,q, with ">="
 *           as in Algorithm 1.  q runs over h, qx=hu, qy=hv and z.
 *  R-reg    regularisation: R1 marks the four children of every
 *           significant detail (levels <= L-2) significant; R2 then marks
 *           every ancestor of a significant detail significant.
 *  R-nbr    neighbours are the same-level cells (Sec. 2.1.3); outside the
 *           domain a ghost copy of the leaf itself is used, with the normal
 *           discharge negated for a closed or inflow side.
 *  R-Lc     L_c (deferred by the paper to Liang 2010): first-order
 *           hydrostatic reconstruction at every face (h* = eta - max(zL,zR)),
 *           HLL flux with two-rarefaction wave-speed estimates and dry-bed
 *           speeds, and the bed-slope source of the same reconstruction,
 *           g/2*(h*_W^2 - h*_E^2)/dx with the cell's own reconstructed
 *           depths at its two faces (Audusse et al. 2004), which keeps a
 *           lake at rest still also next to dry ground; a face side with
 *           reconstructed depth below tol_h is dry (depth 0); cell
 *           velocities are q*(1/h) for h >= tol_h, else 0.  After the
 *           update a negative depth becomes 0 and a cell left below tol_h
 *           loses its discharges.
 *  R-fric   Manning friction by semi-implicit splitting after the flux
 *           update: q <- q * (1/D), D = 1 + dt*g*nM^2*|u|/(h*cbrt(h)).
 *  R-cfl    dt = CFL * min over wet leaves (h >= tol_h) of
 *           min(dx_L/(|u|+sqrt(gh)), dy_L/(|v|+sqrt(gh))) with the finest
 *           spacing dx_L, dy_L and the leaf's updated state (the grid may
 *           refine by one level before the next update), capped at dt_max
 *           (which is also the step when every leaf is dry).  Before the
 *           first step the same formula runs over the finest cells of the
 *           initial state.
 *  R-decode after the update the finest cells under a leaf take the leaf's
 *           discharges (Eq. 4 with the details below leaves set to zero).
 *           Their depth restores the leaf's free surface: with
 *           eta = h_leaf + z_leaf (z_leaf the leaf's bed coefficient), a
 *           finest cell of bed z gets max(0, eta - z).  A leaf on the finest
 *           level, or a dry leaf (h_leaf < tol_h), hands down h_leaf as is.
 *           Handing down h itself would turn a still free surface over an
 *           uneven bed into a sloping one (Sec. 3.1 reports the method
 *           well-balanced), and restoring eta on a dry leaf would create
 *           water in the hollows of the bed.
 *  R-inflow an inflow side is a closed wall plus a volume source
 *           Q(t)*dt*(covered inlet length / inlet length) on every leaf that
 *           touches the inlet, Q piecewise linear in t, taken at the start
 *           of the step.
 *  R-match  (optional, flux_match = 1; the conservative variant the paper
 *           leaves out of its same-level rule, Sec. 2.1.3) a face of a leaf
 *           whose same-level neighbour is refined (significant after R2, so
 *           smaller leaves lie on the other side) does not use that
 *           neighbour's coarse coefficient: its flux and the leaf's own
 *           reconstructed depth squared (the bed source term's face value)
 *           are the averages, 0.5*(first half + second half), of those of
 *           its two half faces one level finer, recursively, down to the
 *           half faces whose neighbour cell is a leaf.  Such a half face is
 *           evaluated between the same-level cells on both sides of it, the
 *           call the smaller leaf makes for the same face, so every face
 *           between leaves of two levels carries one flux from both sides
 *           (mass is conserved up to rounding), and a still free surface
 *           stays still.  Needs R2 (a significant cell then has only
 *           significant ancestors).
 *  R-skip   (the learned subtree skip, a layer the project adds; the paper
 *           has no learned part) each level-(L-4) subtree is encoded,
 *           flagged and stored only down to a given predicted level; the
 *           steps are stated with orc_skip_step below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_VERSION 2

/* ------------------------------------------------------------------------ */
/* Problem description (a plain C struct mirrored by oracle/__init__.py).   */
/* ------------------------------------------------------------------------ */
enum { ORC_BC_CLOSED = 0, ORC_BC_TRANSMISSIVE = 1, ORC_BC_INFLOW = 2 };
enum { ORC_W = 0, ORC_E = 1, ORC_S = 2, ORC_N = 3 };

typedef struct {
    double x0, y0, lx, ly;   /* domain origin and extent (m)               */
    int L;                   /* maximum refinement level                   */
    int reg_predict;         /* R1 on/off                                  */
    int reg_close;           /* R2 on/off                                  */
    int inflow_a0, inflow_a1;/* inlet: finest cells [a0,a1) along the side */
    int inflow_n;            /* number of (t, Q) hydrograph points         */
    int bc[4];               /* W, E, S, N                                 */
    double eps, cfl, g, manning_n, tol_h, dt_max;
    const double* inflow_t;
    const double* inflow_Q;
    int flux_match;          /* R-match on/off                             */
} orc_problem;

int orc_version(void) { return ORC_VERSION; }

/* ------------------------------------------------------------------------ */
/* Indexing: Morton code and hierarchy (Z-order) index, Sec. 2.2.1, Fig. 5. */
/* ------------------------------------------------------------------------ */

/* Morton code of cell (i, j): bit b of i goes to bit 2b, bit b of j to bit
 * 2b+1 (Fig. 5a: interleaving of the binary i and j indices). */
uint64_t orc_morton(uint32_t i, uint32_t j) {
    uint64_t code = 0;
    for (int b = 0; b < 32; ++b) {
        code |= (uint64_t)((i >> b) & 1u) << (2 * b);
        code |= (uint64_t)((j >> b) & 1u) << (2 * b + 1);
    }
    return code;
}

/* Inverse of orc_morton. */
void orc_demorton(uint64_t code, uint32_t* i, uint32_t* j) {
    uint32_t a = 0, b = 0;
    for (int k = 0; k < 32; ++k) {
        a |= (uint32_t)((code >> (2 * k)) & 1u) << k;
        b |= (uint32_t)((code >> (2 * k + 1)) & 1u) << k;
    }
    *i = a;
    *j = b;
}

/* Number of cells in levels 0..n-1, i.e. where level n starts in the
 * hierarchy: 1 + 4 + ... + 4^(n-1) = (4^n - 1)/3. */
static int64_t level_start(int n) {
    int64_t s = 0, c = 1;
    for (int k = 0; k < n; ++k) { s += c; c *= 4; }
    return s;
}

/* Z-order index of a cell in the hierarchy (Sec. 2.2.1, footnote 2): the
 * cells of coarser levels come first, then the Morton code in level n. */
int64_t orc_zindex(int n, uint64_t code) { return level_start(n) + (int64_t)code; }

static int64_t side(int n) { return (int64_t)1 << n; }
static int64_t rm(int n, int64_t i, int64_t j) { return j * side(n) + i; }

/* ------------------------------------------------------------------------ */
/* Haar encoding and decoding, Eq. 3a-3d and Eq. 4a-4d.                     */
/* Children: [0]=(2i,2j) [1]=(2i+1,2j) [2]=(2i,2j+1) [3]=(2i+1,2j+1)          */
/* (the Z-order motif of Fig. 5b).                                          */
/* ------------------------------------------------------------------------ */

/* One parent from its four children (Eq. 3a-3d with taps 1/2, -1/2).  The
 * inner brackets of Eq. 3 pair [0] with [2] and [1] with [3]. */
void orc_encode_parent(const double c[4], double out[4]) {
    double a = c[0] + c[2];       /* H-sum of the first pair   */
    double b = c[1] + c[3];       /* H-sum of the second pair  */
    double d = c[0] - c[2];       /* G-difference, first pair  */
    double e = c[1] - c[3];       /* G-difference, second pair */
    out[0] = 0.25 * (a + b);      /* s      (Eq. 3a) */
    out[1] = 0.25 * (d + e);      /* d_alpha (Eq. 3b) */
    out[2] = 0.25 * (a - b);      /* d_beta  (Eq. 3c) */
    out[3] = 0.25 * (d - e);      /* d_gamma (Eq. 3d) */
}

/* Four children from a parent and its details (Eq. 4a-4d, decode taps
 * 1, 1, 1, -1). */
void orc_decode_parent(const double p[4], double c[4]) {
    double s = p[0], da = p[1], db = p[2], dg = p[3];
    c[0] = (s + da) + (db + dg);  /* Eq. 4a */
    c[2] = (s - da) + (db - dg);  /* Eq. 4b */
    c[1] = (s + da) - (db + dg);  /* Eq. 4c */
    c[3] = (s - da) - (db - dg);  /* Eq. 4d */
}

/* Encoding (Algorithm 1, Eq. 3): from the finest level L (row-major
 * 2^L x 2^L in `fine`) produce every level.  `hier` receives all levels
 * 0..L (level n at level_start(n), row-major).  When `det` is not NULL it
 * receives the three details of every parent (levels 0..L-1), 3 doubles per
 * parent at 3*(level_start(n) + j*2^n + i). */
void orc_encode(int L, const double* fine, double* hier, double* det) {
    memcpy(hier + level_start(L), fine, sizeof(double) * (size_t)(side(L) * side(L)));
    for (int n = L - 1; n >= 0; --n) {           /* Algorithm 1, outer loop */
        const double* ch = hier + level_start(n + 1);
        double* pa = hier + level_start(n);
        for (int64_t j = 0; j < side(n); ++j) {  /* inner loop over cells */
            for (int64_t i = 0; i < side(n); ++i) {
                double c[4], o[4];
                c[0] = ch[rm(n + 1, 2 * i, 2 * j)];
                c[1] = ch[rm(n + 1, 2 * i + 1, 2 * j)];
                c[2] = ch[rm(n + 1, 2 * i, 2 * j + 1)];
                c[3] = ch[rm(n + 1, 2 * i + 1, 2 * j + 1)];
                orc_encode_parent(c, o);
                pa[rm(n, i, j)] = o[0];
                if (det) {
                    int64_t k = 3 * (level_start(n) + rm(n, i, j));
                    det[k] = o[1];
                    det[k + 1] = o[2];
                    det[k + 2] = o[3];
                }
            }
        }
    }
}

/* Full decoding of a hierarchy (Algorithm 4 with every detail applied):
 * rebuild level L from level 0 and all details.  Used to pin the round
 * trip of Eq. 3 / Eq. 4. */
void orc_decode_all(int L, const double* coarse0, const double* det, double* fine_out) {
    double* cur = (double*)malloc(sizeof(double));
    cur[0] = coarse0[0];
    for (int n = 0; n < L; ++n) {
        double* nxt = (double*)malloc(sizeof(double) * (size_t)(side(n + 1) * side(n + 1)));
        for (int64_t j = 0; j < side(n); ++j) {
            for (int64_t i = 0; i < side(n); ++i) {
                int64_t k = 3 * (level_start(n) + rm(n, i, j));
                double p[4] = {cur[rm(n, i, j)], det[k], det[k + 1], det[k + 2]}, c[4];
                orc_decode_parent(p, c);
                nxt[rm(n + 1, 2 * i, 2 * j)] = c[0];
                nxt[rm(n + 1, 2 * i + 1, 2 * j)] = c[1];
                nxt[rm(n + 1, 2 * i, 2 * j + 1)] = c[2];
                nxt[rm(n + 1, 2 * i + 1, 2 * j + 1)] = c[3];
            }
        }
        free(cur);
        cur = nxt;
    }
    memcpy(fine_out, cur, sizeof(double) * (size_t)(side(L) * side(L)));
    free(cur);
}

/* ------------------------------------------------------------------------ */
/* Significance: threshold flags (Sec. 2.1.2, Algorithm 1's test) and       */
/* regularisation (R1, R2).  Flags are bytes, level-major, row-major in a   */
/* level, levels 0..L-1 (P = (4^L-1)/3 entries).                            */
/* ------------------------------------------------------------------------ */

static double absd(double x) { return x < 0.0 ? -x : x; }
static double maxd(double a, double b) { return a > b ? a : b; }

/* s_max of one quantity: max(1, max |s^(L)|) over the finest grid. */
double orc_smax(int L, const double* fine) {
    double m = 1.0;
    for (int64_t k = 0; k < side(L) * side(L); ++k) m = maxd(m, absd(fine[k]));
    return m;
}

/* Threshold test of the parent at hierarchy index p: significant when, for
 * any q, max(|da|,|db|,|dg|) >= thr * s_max,q with thr = 2^(n-L) eps.
 * `det4[q]` are the details of quantity q (layout of orc_encode), q = h,
 * qx, qy, z; `smax4[q]` their s_max. */
static int parent_significant(const double* const* det4, int64_t p, double thr, const double* smax4) {
    int sig = 0;
    for (int q = 0; q < 4; ++q) {
        const double* d = det4[q] + 3 * p;
        double dnorm = maxd(maxd(absd(d[0]), absd(d[1])), absd(d[2]));
        if (dnorm >= thr * smax4[q]) sig = 1;
    }
    return sig;
}

/* Threshold flags of every parent (levels 0..L-1). */
void orc_threshold_flags(int L, double eps, const double* const* det4, const double* smax4,
                         uint8_t* T) {
    for (int n = 0; n < L; ++n) {
        double thr = ldexp(eps, n - L);
        for (int64_t j = 0; j < side(n); ++j)
            for (int64_t i = 0; i < side(n); ++i) {
                int64_t p = level_start(n) + rm(n, i, j);
                T[p] = (uint8_t)parent_significant(det4, p, thr, smax4);
            }
    }
}

/* Regularisation.  R1 (prediction): the children of every significant
 * parent at level n <= L-2 become significant.  R2 (closure): every
 * ancestor of a significant parent becomes significant.  R1 reads only the
 * threshold flags; R2 runs on the result of R1. */
void orc_regularise(int L, int predict, int close, const uint8_t* T, uint8_t* S) {
    int64_t P = level_start(L);
    memcpy(S, T, (size_t)P);
    if (predict) {
        for (int n = 0; n + 1 <= L - 1; ++n) {
            for (int64_t j = 0; j < side(n); ++j)
                for (int64_t i = 0; i < side(n); ++i) {
                    if (!T[level_start(n) + rm(n, i, j)]) continue;
                    for (int k = 0; k < 4; ++k)
                        S[level_start(n + 1) + rm(n + 1, 2 * i + (k & 1), 2 * j + (k >> 1))] = 1;
                }
        }
    }
    if (close) {
        /* walk up from every significant cell, finest parents first */
        for (int n = L - 1; n >= 1; --n) {
            for (int64_t j = 0; j < side(n); ++j)
                for (int64_t i = 0; i < side(n); ++i) {
                    if (!S[level_start(n) + rm(n, i, j)]) continue;
                    S[level_start(n - 1) + rm(n - 1, i / 2, j / 2)] = 1;
                }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Leaf identification.                                                     */
/* Leaves are packed as (level << 28) | Morton code within the level.       */
/* ------------------------------------------------------------------------ */

static uint32_t pack_leaf(int n, int64_t i, int64_t j) {
    return ((uint32_t)n << 28) | (uint32_t)orc_morton((uint32_t)i, (uint32_t)j);
}

typedef struct {
    int L;
    const uint8_t* S;
    uint32_t* out;
    int64_t cap, count;
} dft_ctx;

/* Recursive depth-first traversal of Algorithm 2: a cell is a leaf when
 * its detail is not significant or it is on the finest grid; otherwise the
 * four children are visited in the order [0], [1], [2], [3]. */
static void dft_visit(dft_ctx* ctx, int n, int64_t i, int64_t j) {
    if (n == ctx->L || !ctx->S[level_start(n) + rm(n, i, j)]) {
        if (ctx->count < ctx->cap) ctx->out[ctx->count] = pack_leaf(n, i, j);
        ctx->count++;
        return;
    }
    dft_visit(ctx, n + 1, 2 * i, 2 * j);
    dft_visit(ctx, n + 1, 2 * i + 1, 2 * j);
    dft_visit(ctx, n + 1, 2 * i, 2 * j + 1);
    dft_visit(ctx, n + 1, 2 * i + 1, 2 * j + 1);
}

int64_t orc_leaves_dft(int L, const uint8_t* S, uint32_t* out, int64_t cap) {
    dft_ctx ctx = {L, S, out, cap, 0};
    dft_visit(&ctx, 0, 0, 0);
    return ctx.count;
}

/* Parallel tree traversal of Algorithm 5, written as a plain loop over the
 * finest cells: the "thread" for Morton code m starts at the coarsest cell
 * and moves to the ancestor of m one level finer until it meets a detail
 * that is not significant or reaches the finest grid, then records the
 * Z-order index of the cell where it stopped.  out[m] for m in Morton
 * order. */
void orc_leaves_ptt(int L, const uint8_t* S, int64_t* out) {
    for (uint64_t m = 0; m < (uint64_t)(side(L) * side(L)); ++m) {
        int n = 0;
        for (;;) {
            uint64_t code = m >> (2 * (L - n));
            uint32_t i, j;
            orc_demorton(code, &i, &j);
            if (n == L || !S[level_start(n) + rm(n, i, j)]) {
                out[m] = orc_zindex(n, code);
                break;
            }
            n++;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* FV1 spatial operator L_c (Eq. 1, 2; Sec. 2.1.3 for the neighbours).      */
/* ------------------------------------------------------------------------ */

typedef struct { double h, qx, qy, z; } orc_cell;

/* Cell velocity: q*(1/h) when the cell is wet (h >= tol_h), else 0. */
static void velocity(const orc_cell* c, double tol_h, double* u, double* v) {
    if (c->h >= tol_h) {
        double rh = 1.0 / c->h;
        *u = c->qx * rh;
        *v = c->qy * rh;
    } else {
        *u = 0.0;
        *v = 0.0;
    }
}

/* Two-rarefaction estimate of the star region between the two waves of a
 * face with both sides wet (reading R-Lc): its normal velocity us and
 * celerity as.  It is the exact star state of a Riemann problem whose two
 * waves are rarefactions (the Riemann invariants u + 2a and u - 2a carry
 * it across them). */
void orc_star_estimate(double unL, double aL, double unR, double aR, double* us, double* as) {
    *us = 0.5 * (unL + unR) + aL - aR;
    *as = 0.5 * (aL + aR) + 0.25 * (unL - unR);
}

/* HLL flux across one face whose normal points from side L to side R.
 * un/ut are the normal/tangential velocities of each side; F receives
 * (mass, normal momentum, tangential momentum) fluxes.  hLs/hRs return the
 * reconstructed depths, zf the face bed. */
static void hll_face(double g, double tol_h,
                     double hL, double zL, double unL, double utL,
                     double hR, double zR, double unR, double utR,
                     double F[3], double* hLs_out, double* hRs_out, double* zf_out) {
    double zf = maxd(zL, zR);
    double dL = (hL + zL) - zf;                 /* eta_L - z_face */
    double dR = (hR + zR) - zf;
    double hLs = dL >= tol_h ? dL : 0.0;        /* hydrostatic reconstruction */
    double hRs = dR >= tol_h ? dR : 0.0;
    *hLs_out = hLs;
    *hRs_out = hRs;
    *zf_out = zf;
    if (hLs == 0.0 && hRs == 0.0) {
        F[0] = F[1] = F[2] = 0.0;
        return;
    }
    double aL = sqrt(g * hLs), aR = sqrt(g * hRs);
    double SL, SR;
    if (hLs > 0.0 && hRs > 0.0) {               /* two-rarefaction estimate */
        double us, as;
        orc_star_estimate(unL, aL, unR, aR, &us, &as);
        double a1 = unL - aL, a2 = us - as;
        double b1 = unR + aR, b2 = us + as;
        SL = a1 < a2 ? a1 : a2;
        SR = b1 > b2 ? b1 : b2;
    } else if (hLs == 0.0) {                    /* dry bed on the left */
        SL = unR - 2.0 * aR;
        SR = unR + aR;
    } else {                                    /* dry bed on the right */
        SL = unL - aL;
        SR = unL + 2.0 * aL;
    }
    double qnL = hLs * unL, qtL = hLs * utL;
    double qnR = hRs * unR, qtR = hRs * utR;
    double FL0 = qnL, FL1 = qnL * unL + 0.5 * g * hLs * hLs, FL2 = qnL * utL;
    double FR0 = qnR, FR1 = qnR * unR + 0.5 * g * hRs * hRs, FR2 = qnR * utR;
    if (SL >= 0.0) {
        F[0] = FL0; F[1] = FL1; F[2] = FL2;
    } else if (SR <= 0.0) {
        F[0] = FR0; F[1] = FR1; F[2] = FR2;
    } else {
        double inv = 1.0 / (SR - SL);
        F[0] = (SR * FL0 - SL * FR0 + SL * SR * (hRs - hLs)) * inv;
        F[1] = (SR * FL1 - SL * FR1 + SL * SR * (qnR - qnL)) * inv;
        F[2] = (SR * FL2 - SL * FR2 + SL * SR * (qtR - qtL)) * inv;
    }
}

/* Exposed for the flux pins in the tests: x-direction HLL flux between two
 * cell states given as (h, qx, qy, z). */
void orc_hll_x(double g, double tol_h, const double* Lst, const double* Rst, double F[3]) {
    orc_cell a = {Lst[0], Lst[1], Lst[2], Lst[3]}, b = {Rst[0], Rst[1], Rst[2], Rst[3]};
    double uL, vL, uR, vR, hl, hr, zf;
    velocity(&a, tol_h, &uL, &vL);
    velocity(&b, tol_h, &uR, &vR);
    hll_face(g, tol_h, a.h, a.z, uL, vL, b.h, b.z, uR, vR, F, &hl, &hr, &zf);
}

/* Piecewise-linear inflow hydrograph Q(t). */
static double inflow_Q(const orc_problem* p, double t) {
    int n = p->inflow_n;
    if (n <= 0) return 0.0;
    if (t <= p->inflow_t[0]) return p->inflow_Q[0];
    if (t >= p->inflow_t[n - 1]) return p->inflow_Q[n - 1];
    int k = 0;
    while (!(t >= p->inflow_t[k] && t < p->inflow_t[k + 1])) k++;
    double w = (t - p->inflow_t[k]) / (p->inflow_t[k + 1] - p->inflow_t[k]);
    return p->inflow_Q[k] + (p->inflow_Q[k + 1] - p->inflow_Q[k]) * w;
}

/* Ghost state across side `s` of a cell: a copy of the cell, with the
 * normal discharge negated when the side is a wall (closed or inflow). */
static orc_cell ghost(const orc_problem* p, int s, orc_cell c) {
    if (p->bc[s] != ORC_BC_TRANSMISSIVE) {
        if (s == ORC_W || s == ORC_E) c.qx = -c.qx;
        else c.qy = -c.qy;
    }
    return c;
}

/* One face of a cell, seen from the cell: side s (W, E, S, N) between the
 * cell state C and the state X across the face.  F receives the face flux
 * in the order of cell_update (x faces (h, qx, qy), y faces (h, qy, qx)),
 * own2 the square of the cell's own reconstructed depth at the face. */
static void face_of(const orc_problem* p, int s, orc_cell C, orc_cell X, double F[3], double* own2) {
    double g = p->g, tol = p->tol_h;
    double uC, vC, uX, vX, hl, hr, zf;
    velocity(&C, tol, &uC, &vC);
    velocity(&X, tol, &uX, &vX);
    if (s == ORC_W) {               /* X on the left, normal u */
        hll_face(g, tol, X.h, X.z, uX, vX, C.h, C.z, uC, vC, F, &hl, &hr, &zf);
        *own2 = hr * hr;
    } else if (s == ORC_E) {        /* X on the right, normal u */
        hll_face(g, tol, C.h, C.z, uC, vC, X.h, X.z, uX, vX, F, &hl, &hr, &zf);
        *own2 = hl * hl;
    } else if (s == ORC_S) {        /* X below, normal v */
        hll_face(g, tol, X.h, X.z, vX, uX, C.h, C.z, vC, uC, F, &hl, &hr, &zf);
        *own2 = hr * hr;
    } else {                        /* X above, normal v */
        hll_face(g, tol, C.h, C.z, vC, uC, X.h, X.z, vX, uX, F, &hl, &hr, &zf);
        *own2 = hl * hl;
    }
}

/* One FV1 forward-Euler update (Eq. 2) of a cell of size dx x dy from its
 * state C, its four face fluxes (order of face_of) and the squares of its
 * own reconstructed depths at them.  dh_in is the inflow depth added this
 * step (0 when the cell is not on an inlet); `inlet` says whether it is. */
static void cell_update_faces(const orc_problem* p, double dx, double dy, double dt, orc_cell C,
                              const double FW[3], const double FE[3], const double GS[3],
                              const double GN[3], double hW2, double hE2, double hS2, double hN2,
                              int inlet, double dh_in, double out[3]) {
    double g = p->g, tol = p->tol_h;
    double rx = dt / dx, ry = dt / dy;
    /* bed slope from the cell's own reconstructed face depths */
    double bx = 0.5 * g * (hW2 - hE2);
    double by = 0.5 * g * (hS2 - hN2);

    double h = C.h - rx * (FE[0] - FW[0]) - ry * (GN[0] - GS[0]);
    double qx = C.qx - rx * ((FE[1] - FW[1]) + bx) - ry * (GN[2] - GS[2]);
    double qy = C.qy - rx * (FE[2] - FW[2]) - ry * ((GN[1] - GS[1]) + by);
    if (inlet) h = h + dh_in;
    h = h > 0.0 ? h : 0.0;                             /* positivity */
    if (h < tol) {
        qx = 0.0;
        qy = 0.0;
    } else if (p->manning_n > 0.0) {                   /* R-fric */
        double rh = 1.0 / h;
        double u = qx * rh, v = qy * rh;
        double speed = sqrt(u * u + v * v);
        double nM = p->manning_n;
        double D = 1.0 + dt * g * nM * nM * speed / (h * cbrt(h));
        double rD = 1.0 / D;
        qx = qx * rD;
        qy = qy * rD;
    }
    out[0] = h;
    out[1] = qx;
    out[2] = qy;
}

/* The update of a cell from its state and its four same-level neighbour
 * states W, E, S, N (ghosts already applied). */
static void cell_update(const orc_problem* p, double dx, double dy, double dt,
                        orc_cell C, orc_cell W, orc_cell E, orc_cell S, orc_cell N,
                        int inlet, double dh_in, double out[3]) {
    double FW[3], FE[3], GS[3], GN[3], hW2, hE2, hS2, hN2;
    face_of(p, ORC_W, C, W, FW, &hW2);
    face_of(p, ORC_E, C, E, FE, &hE2);
    face_of(p, ORC_S, C, S, GS, &hS2);
    face_of(p, ORC_N, C, N, GN, &hN2);
    cell_update_faces(p, dx, dy, dt, C, FW, FE, GS, GN, hW2, hE2, hS2, hN2, inlet, dh_in, out);
}

/* Read the same-level cell (n, i, j) from the hierarchies. */
static orc_cell fetch(const double* const* hier4, int n, int64_t i, int64_t j) {
    int64_t k = level_start(n) + rm(n, i, j);
    orc_cell c = {hier4[0][k], hier4[1][k], hier4[2][k], hier4[3][k]};
    return c;
}

/* Inflow depth for the leaf (n, i, j) of size dx x dy and whether the leaf
 * touches the inlet. */
static double inflow_depth(const orc_problem* p, int n, int64_t i, int64_t j, double dx,
                           double dy, double t, double dt, int* inlet) {
    *inlet = 0;
    int s = -1;
    for (int k = 0; k < 4; ++k)
        if (p->bc[k] == ORC_BC_INFLOW) s = k;
    if (s < 0 || p->inflow_n <= 0 || p->inflow_a1 <= p->inflow_a0) return 0.0;
    int64_t last = side(n) - 1, a;
    if (s == ORC_W) { if (i != 0) return 0.0; a = j; }
    else if (s == ORC_E) { if (i != last) return 0.0; a = j; }
    else if (s == ORC_S) { if (j != 0) return 0.0; a = i; }
    else { if (j != last) return 0.0; a = i; }
    int64_t w = side(p->L - n);                 /* finest cells per leaf side */
    int64_t lo = a * w, hi = lo + w;
    if (lo < p->inflow_a0) lo = p->inflow_a0;
    if (hi > p->inflow_a1) hi = p->inflow_a1;
    if (hi <= lo) return 0.0;
    *inlet = 1;
    double frac = (double)(hi - lo) / (double)(p->inflow_a1 - p->inflow_a0);
    double Q = inflow_Q(p, t);
    return ((Q * dt) * frac) / (dx * dy);
}

/* Whether the cell (n, i, j) is refined: below the finest level and
 * significant after regularisation. */
static int refined(const orc_problem* p, const uint8_t* S, int n, int64_t i, int64_t j) {
    return n < p->L && S[level_start(n) + rm(n, i, j)];
}

/* R-match: the face on side s of the cell (n, i, j) whose neighbour cell
 * (n, ni, nj) across that face is refined.  The face splits into two half
 * faces one level finer; on each, the own-side cell and the neighbour
 * cell are the level-(n+1) children that touch it (own side: the children
 * of (n, i, j) next to the face; neighbour side: those of (n, ni, nj)).
 * A half face whose neighbour child is refined again is split again. */
static void matched_face(const orc_problem* p, const double* const* hier4, const uint8_t* S, int s,
                         int n, int64_t i, int64_t j, int64_t ni, int64_t nj, double F[3],
                         double* own2) {
    double Fa[3], Fb[3], oa, ob;
    for (int half = 0; half < 2; ++half) {
        int64_t ci, cj, cni, cnj;            /* children at level n+1 */
        if (s == ORC_W || s == ORC_E) {      /* x face: the halves go up in j */
            ci = 2 * i + (s == ORC_E ? 1 : 0);
            cni = 2 * ni + (s == ORC_E ? 0 : 1);
            cj = cnj = 2 * j + half;
        } else {                             /* y face: the halves go along i */
            cj = 2 * j + (s == ORC_N ? 1 : 0);
            cnj = 2 * nj + (s == ORC_N ? 0 : 1);
            ci = cni = 2 * i + half;
        }
        double* Fh = half ? Fb : Fa;
        double* oh = half ? &ob : &oa;
        if (refined(p, S, n + 1, cni, cnj))
            matched_face(p, hier4, S, s, n + 1, ci, cj, cni, cnj, Fh, oh);
        else
            face_of(p, s, fetch(hier4, n + 1, ci, cj), fetch(hier4, n + 1, cni, cnj), Fh, oh);
    }
    for (int k = 0; k < 3; ++k) F[k] = 0.5 * (Fa[k] + Fb[k]);
    *own2 = 0.5 * (oa + ob);
}

/* One face of the leaf (n, i, j) on side s: the ghost at the domain edge,
 * else the same-level neighbour (Sec. 2.1.3, Fig. 3), or with R-match the
 * averaged finer faces when that neighbour is refined. */
static void leaf_face(const orc_problem* p, const double* const* hier4, const uint8_t* S, int s,
                      int n, int64_t i, int64_t j, orc_cell C, double F[3], double* own2) {
    int64_t last = side(n) - 1;
    int64_t ni = i + (s == ORC_E) - (s == ORC_W), nj = j + (s == ORC_N) - (s == ORC_S);
    if (ni < 0 || ni > last || nj < 0 || nj > last) {
        face_of(p, s, C, ghost(p, s, C), F, own2);
    } else if (p->flux_match && refined(p, S, n, ni, nj)) {
        matched_face(p, hier4, S, s, n, i, j, ni, nj, F, own2);
    } else {
        face_of(p, s, C, fetch(hier4, n, ni, nj), F, own2);
    }
}

/* FV1 update of one leaf (n, i, j) using same-level neighbours from the
 * hierarchies (Sec. 2.1.3, Fig. 3); S the regularised flags (read by
 * R-match only). */
static void leaf_update(const orc_problem* p, const double* const* hier4, const uint8_t* S, int n,
                        int64_t i, int64_t j, double t, double dt, double out[3]) {
    double dx = ldexp(p->lx, -n), dy = ldexp(p->ly, -n);
    orc_cell C = fetch(hier4, n, i, j);
    double FW[3], FE[3], GS[3], GN[3], hW2, hE2, hS2, hN2;
    leaf_face(p, hier4, S, ORC_W, n, i, j, C, FW, &hW2);
    leaf_face(p, hier4, S, ORC_E, n, i, j, C, FE, &hE2);
    leaf_face(p, hier4, S, ORC_S, n, i, j, C, GS, &hS2);
    leaf_face(p, hier4, S, ORC_N, n, i, j, C, GN, &hN2);
    int inlet;
    double dh = inflow_depth(p, n, i, j, dx, dy, t, dt, &inlet);
    cell_update_faces(p, dx, dy, dt, C, FW, FE, GS, GN, hW2, hE2, hS2, hN2, inlet, dh, out);
}

/* CFL bound of one cell state (R-cfl): min(dx/(|u|+a), dy/(|v|+a)) with
 * the finest spacings, or +inf for a dry cell. */
static double cfl_bound(const orc_problem* p, double h, double qx, double qy) {
    if (h < p->tol_h) return INFINITY;
    double dx = ldexp(p->lx, -p->L), dy = ldexp(p->ly, -p->L);
    double rh = 1.0 / h;
    double u = absd(qx * rh), v = absd(qy * rh);
    double a = sqrt(p->g * h);
    double rx = dx / (u + a), ry = dy / (v + a);
    return rx < ry ? rx : ry;
}

/* CFL reduction over the finest grid: min of cfl_bound, +inf if all dry. */
double orc_cfl_rmin(const orc_problem* p, const double* h, const double* qx, const double* qy) {
    double r = INFINITY;
    for (int64_t k = 0; k < side(p->L) * side(p->L); ++k) {
        double rr = cfl_bound(p, h[k], qx[k], qy[k]);
        if (rr < r) r = rr;
    }
    return r;
}

static double dt_from_rmin(const orc_problem* p, double r) {
    double dt = p->cfl * r;                 /* +inf when every cell is dry */
    return dt < p->dt_max ? dt : p->dt_max;
}

/* dt from the finest cells of a state (used before the first step). */
double orc_next_dt(const orc_problem* p, const double* h, const double* qx, const double* qy) {
    return dt_from_rmin(p, orc_cfl_rmin(p, h, qx, qy));
}

/* ------------------------------------------------------------------------ */
/* One HWFV1 timestep (Algorithm 3, the body of its time loop).             */
/* ------------------------------------------------------------------------ */

typedef struct {
    /* optional outputs, each may be NULL */
    uint8_t* T;          /* threshold flags, P bytes                       */
    uint8_t* S;          /* regularised flags, P bytes                     */
    uint32_t* leaves;    /* packed leaves, capacity leaves_cap             */
    int64_t leaves_cap;
    double* hier_out;    /* 3*(N+P): encoded h, qx, qy of every level      */
    /* scalar outputs */
    int64_t num_leaves;
    double dt_next;
} orc_step_out;

/* Advance the finest state (h, qx, qy row-major, in place) by one step of
 * size dt starting at time t.  z is the finest bed.  Returns 0 on success.
 * The step is: encode h, qx, qy, z (Algorithm 1); flag and regularise;
 * find the leaves by DFT (Algorithm 2); FV1-update every leaf from its
 * same-level neighbours (Sec. 2.1.3); put the new leaf values on the finest
 * grid (R-decode); compute the next dt (R-cfl). */
static int hwfv1_step_smax(const orc_problem* p, double* h, double* qx, double* qy, const double* z,
                           double t, double dt, const double* smax_in, orc_step_out* o);

int orc_hwfv1_step(const orc_problem* p, double* h, double* qx, double* qy, const double* z,
                   double t, double dt, orc_step_out* o) {
    return hwfv1_step_smax(p, h, qx, qy, z, t, dt, NULL, o);
}

/* The step with the s_max of h, qx, qy given (smax_in, 3 values) instead of
 * taken over the finest fields; NULL takes them over the finest fields. */
static int hwfv1_step_smax(const orc_problem* p, double* h, double* qx, double* qy, const double* z,
                           double t, double dt, const double* smax_in, orc_step_out* o) {
    int L = p->L;
    if (p->flux_match && !p->reg_close) return 2;     /* R-match needs R2 */
    int64_t N = side(L) * side(L), P = level_start(L), H = N + P;
    double* hier[4];
    double* det[4];
    const double* fine[4] = {h, qx, qy, z};
    double smax[4];
    for (int q = 0; q < 4; ++q) {
        hier[q] = (double*)malloc(sizeof(double) * (size_t)H);
        det[q] = (double*)malloc(sizeof(double) * (size_t)(3 * (P > 0 ? P : 1)));
        if (!hier[q] || !det[q]) return 1;
        orc_encode(L, fine[q], hier[q], det[q]);
        smax[q] = (smax_in && q < 3) ? smax_in[q] : orc_smax(L, fine[q]);
    }
    uint8_t* T = (uint8_t*)malloc((size_t)(P > 0 ? P : 1));
    uint8_t* S = (uint8_t*)malloc((size_t)(P > 0 ? P : 1));
    orc_threshold_flags(L, p->eps, (const double* const*)det, smax, T);
    orc_regularise(L, p->reg_predict, p->reg_close, T, S);

    int64_t M = orc_leaves_dft(L, S, NULL, 0);
    uint32_t* leaves = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)M);
    orc_leaves_dft(L, S, leaves, M);

    double* newU = (double*)malloc(sizeof(double) * (size_t)(3 * M));
    for (int64_t k = 0; k < M; ++k) {
        int n = (int)(leaves[k] >> 28);
        uint32_t i, j;
        orc_demorton(leaves[k] & 0x0FFFFFFFu, &i, &j);
        leaf_update(p, (const double* const*)hier, S, n, i, j, t, dt, newU + 3 * k);
    }
    /* R-cfl over the updated leaves */
    double rmin = INFINITY;
    for (int64_t k = 0; k < M; ++k) {
        double rr = cfl_bound(p, newU[3 * k], newU[3 * k + 1], newU[3 * k + 2]);
        if (rr < rmin) rmin = rr;
    }
    /* R-decode: the finest cells under a leaf take its discharges and, on a
     * wet coarse leaf, its free surface */
    for (int64_t k = 0; k < M; ++k) {
        int n = (int)(leaves[k] >> 28);
        uint32_t i, j;
        orc_demorton(leaves[k] & 0x0FFFFFFFu, &i, &j);
        int64_t w = side(L - n);
        double hl = newU[3 * k];
        int restore = n < L && hl >= p->tol_h;
        double eta = restore ? hl + hier[3][level_start(n) + rm(n, i, j)] : 0.0;
        for (int64_t jj = j * w; jj < (j + 1) * w; ++jj)
            for (int64_t ii = i * w; ii < (i + 1) * w; ++ii) {
                double hf = hl;
                if (restore) {
                    double d = eta - z[rm(L, ii, jj)];
                    hf = d > 0.0 ? d : 0.0;
                }
                h[rm(L, ii, jj)] = hf;
                qx[rm(L, ii, jj)] = newU[3 * k + 1];
                qy[rm(L, ii, jj)] = newU[3 * k + 2];
            }
    }
    if (o) {
        if (o->T) memcpy(o->T, T, (size_t)P);
        if (o->S) memcpy(o->S, S, (size_t)P);
        if (o->leaves) memcpy(o->leaves, leaves, sizeof(uint32_t) * (size_t)(M < o->leaves_cap ? M : o->leaves_cap));
        if (o->hier_out)
            for (int q = 0; q < 3; ++q) memcpy(o->hier_out + q * H, hier[q], sizeof(double) * (size_t)H);
        o->num_leaves = M;
        o->dt_next = dt_from_rmin(p, rmin);
    }
    for (int q = 0; q < 4; ++q) { free(hier[q]); free(det[q]); }
    free(T); free(S); free(leaves); free(newU);
    return 0;
}

/* One uniform-grid FV1 step on the finest grid (the GPU-FV1 stand-in):
 * every finest cell is updated from its finest neighbours. */
int orc_fv1_step(const orc_problem* p, double* h, double* qx, double* qy, const double* z,
                 double t, double dt) {
    int L = p->L;
    int64_t N = side(L) * side(L), last = side(L) - 1;
    double* nu = (double*)malloc(sizeof(double) * (size_t)(3 * N));
    if (!nu) return 1;
    double dx = ldexp(p->lx, -L), dy = ldexp(p->ly, -L);
#define CELL(ii, jj) ((orc_cell){h[rm(L, ii, jj)], qx[rm(L, ii, jj)], qy[rm(L, ii, jj)], z[rm(L, ii, jj)]})
    for (int64_t j = 0; j <= last; ++j)
        for (int64_t i = 0; i <= last; ++i) {
            orc_cell C = CELL(i, j);
            orc_cell W = i > 0 ? CELL(i - 1, j) : ghost(p, ORC_W, C);
            orc_cell E = i < last ? CELL(i + 1, j) : ghost(p, ORC_E, C);
            orc_cell S = j > 0 ? CELL(i, j - 1) : ghost(p, ORC_S, C);
            orc_cell Nn = j < last ? CELL(i, j + 1) : ghost(p, ORC_N, C);
            int inlet;
            double dh = inflow_depth(p, L, i, j, dx, dy, t, dt, &inlet);
            cell_update(p, dx, dy, dt, C, W, E, S, Nn, inlet, dh, nu + 3 * rm(L, i, j));
        }
#undef CELL
    for (int64_t k = 0; k < N; ++k) {
        h[k] = nu[3 * k];
        qx[k] = nu[3 * k + 1];
        qy[k] = nu[3 * k + 2];
    }
    free(nu);
    return 0;
}

/* Time loop of Algorithm 3: advance until t_end or max_steps.  `uniform`
 * selects plain FV1 on the finest grid instead of HWFV1.  On entry *t and
 * *dt hold the current time and the step to take next; on exit they hold
 * the final values.  *steps and *leaf_updates accumulate counts. */
int orc_run(const orc_problem* p, double* h, double* qx, double* qy, const double* z,
            double* t, double* dt, double t_end, int64_t max_steps, int uniform,
            int64_t* steps, int64_t* leaf_updates) {
    for (int64_t s = 0; s < max_steps && *t < t_end; ++s) {
        double dt_use = *dt;
        if (*t + dt_use > t_end) dt_use = t_end - *t;
        if (uniform) {
            if (orc_fv1_step(p, h, qx, qy, z, *t, dt_use)) return 1;
            *leaf_updates += (int64_t)1 << (2 * p->L);
            *t = *t + dt_use;
            *dt = orc_next_dt(p, h, qx, qy);
        } else {
            orc_step_out o;
            memset(&o, 0, sizeof o);
            if (orc_hwfv1_step(p, h, qx, qy, z, *t, dt_use, &o)) return 1;
            *leaf_updates += o.num_leaves;
            *t = *t + dt_use;
            *dt = o.dt_next;
        }
        *steps += 1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Learned subtree skip: the project's learned layer on Algorithm 3         */
/* (reading R-skip; the paper has no learned part).                         */
/*                                                                          */
/* The subtrees are the cells of level Ls = L - 4 (16 x 16 finest cells     */
/* each).  Subtree s keeps its state at a storage level m_s, Ls <= m_s <= L: */
/* the values of its level-m_s cells (m_s = L at the start and after every  */
/* plain step).  A skip step is given a level p_s in [Ls, L] per subtree    */
/* (the prediction of the deepest level the subtree needs) and              */
/*  1. takes P_s = max(p_s, p of the subtrees sharing an edge with s): the  */
/*     level s is kept down to, so that a leaf of a neighbouring subtree    */
/*     (no finer than its own p) finds its same-level neighbour cells in s; */
/*  2. takes s_max,q = max(1, max |value|) over the stored state (the       */
/*     level-m_s cells of every subtree) as it is when the step starts;     */
/*  3. when P_s > m_s, forms the level-P_s cells of s from its level-m_s    */
/*     cells as the decode-back forms the cells under a leaf (R-decode,     */
/*     with the level-m_s cell as the leaf and z^(P_s) below it);           */
/*  4. encodes s from level E_s = max(m_s, P_s) up to level Ls (Eq. 3), and */
/*     the levels Ls-1 .. 0 from level Ls;                                  */
/*  5. flags a parent (n, c) as the plain step does (q over h, qx, qy, z)   */
/*     when n < Ls, and when n >= Ls only if n < p_s: the subtree's details */
/*     at levels >= p_s are neither used nor tested;                        */
/*  6. regularises (R1, R2) and then clears every cell of a level n >= Ls   */
/*     with n >= p_s, so the leaves of s are no finer than p_s;             */
/*  7. finds the leaves (Algorithm 2) and updates them from their           */
/*     same-level neighbours (Sec. 2.1.3) as the plain step does, with the  */
/*     finest spacing in the CFL bound (R-cfl);                             */
/*  8. stores s at level P_s: every level-P_s cell takes its covering       */
/*     leaf's new value, with the R-decode free surface against z^(P_s)     */
/*     when the leaf is coarser than P_s; then m_s = P_s.                   */
/* A plain step (the exact audit) takes s_max as in 2, forms level L of     */
/* every subtree as in 3, then runs the plain step on the finest grid.      */
/* State layout: h, qx, qy each a full hierarchy (levels 0..L, level n at   */
/* level_start(n), row-major); m and p row-major over level Ls.             */
/* ------------------------------------------------------------------------ */

/* Level-P cells of subtree (si, sj) from its level-m cells, m < P (step 3). */
static void skip_prolong(const orc_problem* p, double* const* hier3, const double* zh, int Ls,
                         int64_t si, int64_t sj, int m, int P) {
    int64_t w = side(P - Ls);                   /* level-P cells per subtree side */
    for (int64_t jj = sj * w; jj < (sj + 1) * w; ++jj)
        for (int64_t ii = si * w; ii < (si + 1) * w; ++ii) {
            int64_t ai = ii >> (P - m), aj = jj >> (P - m);
            int64_t ka = level_start(m) + rm(m, ai, aj), kc = level_start(P) + rm(P, ii, jj);
            double hl = hier3[0][ka];
            double hf = hl;
            if (hl >= p->tol_h) {
                double eta = hl + zh[ka];
                double d = eta - zh[kc];
                hf = d > 0.0 ? d : 0.0;
            }
            hier3[0][kc] = hf;
            hier3[1][kc] = hier3[1][ka];
            hier3[2][kc] = hier3[2][ka];
        }
}

/* Every subtree stored above level L is brought to level L (step 3 with
 * P = L), for the plain step and for reading the finest fields. */
int orc_skip_prolong_all(const orc_problem* p, double* const* hier3, uint8_t* m, const double* z) {
    int L = p->L, Ls = L - 4;
    if (Ls < 0) return 2;
    double* zh = (double*)malloc(sizeof(double) * (size_t)level_start(L + 1));
    if (!zh) return 1;
    orc_encode(L, z, zh, NULL);
    for (int64_t sj = 0; sj < side(Ls); ++sj)
        for (int64_t si = 0; si < side(Ls); ++si) {
            uint8_t* ms = &m[rm(Ls, si, sj)];
            if (*ms < L) skip_prolong(p, hier3, zh, Ls, si, sj, *ms, L);
            *ms = (uint8_t)L;
        }
    free(zh);
    return 0;
}

/* s_max of h, qx, qy over the stored state (the level-m_s cells of every
 * subtree), floored at 1 (R-norm). */
static void skip_smax(const double* const* hier3, const uint8_t* m, int Ls, double smax3[3]) {
    smax3[0] = smax3[1] = smax3[2] = 1.0;
    for (int64_t sj = 0; sj < side(Ls); ++sj)
        for (int64_t si = 0; si < side(Ls); ++si) {
            int ms = m[rm(Ls, si, sj)];
            int64_t w = side(ms - Ls);
            for (int64_t jj = sj * w; jj < (sj + 1) * w; ++jj)
                for (int64_t ii = si * w; ii < (si + 1) * w; ++ii)
                    for (int q = 0; q < 3; ++q)
                        smax3[q] = maxd(smax3[q], absd(hier3[q][level_start(ms) + rm(ms, ii, jj)]));
        }
}

/* The plain step (the exact audit) from a skip state: s_max over the stored
 * state as the step starts, every subtree brought to level L, then the
 * plain step on the finest grid (level L of the hierarchies, in place). */
int orc_skip_audit_step(const orc_problem* p, double* const* hier3, uint8_t* m, const double* z,
                        double t, double dt, orc_step_out* o) {
    int L = p->L, Ls = L - 4;
    if (Ls < 0) return 2;
    double smax3[3];
    skip_smax((const double* const*)hier3, m, Ls, smax3);
    int rc = orc_skip_prolong_all(p, hier3, m, z);
    if (rc) return rc;
    int64_t f0 = level_start(L);
    return hwfv1_step_smax(p, hier3[0] + f0, hier3[1] + f0, hier3[2] + f0, z, t, dt, smax3, o);
}

/* Subtree (row-major index at level Ls) of the cell (n, i, j), n >= Ls. */
static int64_t subtree_of(int Ls, int n, int64_t i, int64_t j) {
    return rm(Ls, i >> (n - Ls), j >> (n - Ls));
}

/* One skip step of size dt at time t (steps 1-8 above).  `pred` holds p_s.
 * Returns 0 on success, 2 for an unsupported problem (L < 4, R-match, or
 * the regularisation not fully on), 3 for a level outside [Ls, L]. */
int orc_skip_step(const orc_problem* p, double* const* hier3, uint8_t* m, const uint8_t* pred,
                  const double* z, double t, double dt, orc_step_out* o) {
    int L = p->L, Ls = L - 4;
    if (Ls < 0 || p->flux_match || !p->reg_predict || !p->reg_close) return 2;
    int64_t ns = side(Ls), NSUB = ns * ns, P_ = level_start(L), H = level_start(L + 1);
    for (int64_t k = 0; k < NSUB; ++k)
        if (pred[k] < Ls || pred[k] > L || m[k] < Ls || m[k] > L) return 3;
    /* 1. storage level of each subtree */
    uint8_t* P = (uint8_t*)malloc((size_t)NSUB);
    for (int64_t sj = 0; sj < ns; ++sj)
        for (int64_t si = 0; si < ns; ++si) {
            int v = pred[rm(Ls, si, sj)];
            if (si > 0 && pred[rm(Ls, si - 1, sj)] > v) v = pred[rm(Ls, si - 1, sj)];
            if (si < ns - 1 && pred[rm(Ls, si + 1, sj)] > v) v = pred[rm(Ls, si + 1, sj)];
            if (sj > 0 && pred[rm(Ls, si, sj - 1)] > v) v = pred[rm(Ls, si, sj - 1)];
            if (sj < ns - 1 && pred[rm(Ls, si, sj + 1)] > v) v = pred[rm(Ls, si, sj + 1)];
            P[rm(Ls, si, sj)] = (uint8_t)v;
        }
    /* 2. s_max over the stored state */
    double smax[4];
    skip_smax((const double* const*)hier3, m, Ls, smax);
    smax[3] = orc_smax(L, z);
    /* the bed: every level and detail (static) */
    double* zh = (double*)malloc(sizeof(double) * (size_t)H);
    double* zdet = (double*)malloc(sizeof(double) * (size_t)(3 * (P_ > 0 ? P_ : 1)));
    orc_encode(L, z, zh, zdet);
    /* 3. prolongation where P_s > m_s; E_s = max(m_s, P_s) */
    uint8_t* E = (uint8_t*)malloc((size_t)NSUB);
    for (int64_t sj = 0; sj < ns; ++sj)
        for (int64_t si = 0; si < ns; ++si) {
            int64_t s = rm(Ls, si, sj);
            if (P[s] > m[s]) skip_prolong(p, hier3, zh, Ls, si, sj, m[s], P[s]);
            E[s] = P[s] > m[s] ? P[s] : m[s];
        }
    /* 4. encode: inside each subtree from level E_s, then above Ls */
    double* det[3];
    for (int q = 0; q < 3; ++q) det[q] = (double*)calloc((size_t)(3 * (P_ > 0 ? P_ : 1)), sizeof(double));
    for (int n = L - 1; n >= 0; --n)
        for (int64_t j = 0; j < side(n); ++j)
            for (int64_t i = 0; i < side(n); ++i) {
                if (n >= Ls && n >= E[subtree_of(Ls, n, i, j)]) continue;  /* level n+1 not formed */
                for (int q = 0; q < 3; ++q) {
                    const double* kid = hier3[q] + level_start(n + 1);
                    double c[4] = {kid[rm(n + 1, 2 * i, 2 * j)], kid[rm(n + 1, 2 * i + 1, 2 * j)],
                                   kid[rm(n + 1, 2 * i, 2 * j + 1)], kid[rm(n + 1, 2 * i + 1, 2 * j + 1)]};
                    double out[4];
                    orc_encode_parent(c, out);
                    int64_t k = level_start(n) + rm(n, i, j);
                    hier3[q][k] = out[0];
                    det[q][3 * k] = out[1];
                    det[q][3 * k + 1] = out[2];
                    det[q][3 * k + 2] = out[3];
                }
            }
    /* 5. threshold flags of the parents allowed to refine */
    uint8_t* T = (uint8_t*)calloc((size_t)(P_ > 0 ? P_ : 1), 1);
    uint8_t* S = (uint8_t*)calloc((size_t)(P_ > 0 ? P_ : 1), 1);
    const double* det4[4] = {det[0], det[1], det[2], zdet};
    for (int n = 0; n < L; ++n) {
        double thr = ldexp(p->eps, n - L);
        for (int64_t j = 0; j < side(n); ++j)
            for (int64_t i = 0; i < side(n); ++i) {
                if (n >= Ls && n >= pred[subtree_of(Ls, n, i, j)]) continue;
                int64_t k = level_start(n) + rm(n, i, j);
                T[k] = (uint8_t)parent_significant(det4, k, thr, smax);
            }
    }
    /* 6. regularisation, then no leaf of s finer than p_s */
    orc_regularise(L, 1, 1, T, S);
    for (int n = Ls; n < L; ++n)
        for (int64_t j = 0; j < side(n); ++j)
            for (int64_t i = 0; i < side(n); ++i)
                if (n >= pred[subtree_of(Ls, n, i, j)]) S[level_start(n) + rm(n, i, j)] = 0;
    /* 7. leaves and their update */
    int64_t M = orc_leaves_dft(L, S, NULL, 0);
    uint32_t* leaves = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(M > 0 ? M : 1));
    orc_leaves_dft(L, S, leaves, M);
    double* newU = (double*)malloc(sizeof(double) * (size_t)(3 * (M > 0 ? M : 1)));
    const double* hier4[4] = {hier3[0], hier3[1], hier3[2], zh};
    for (int64_t k = 0; k < M; ++k) {
        int n = (int)(leaves[k] >> 28);
        uint32_t i, j;
        orc_demorton(leaves[k] & 0x0FFFFFFFu, &i, &j);
        leaf_update(p, hier4, S, n, i, j, t, dt, newU + 3 * k);
    }
    double rmin = INFINITY;
    for (int64_t k = 0; k < M; ++k) {
        double rr = cfl_bound(p, newU[3 * k], newU[3 * k + 1], newU[3 * k + 2]);
        if (rr < rmin) rmin = rr;
    }
    /* 8. store each subtree at level P_s: the leaves' new values at their
     * own cells first (a map from cell to value), then every level-P_s
     * cell from its covering leaf */
    double* nv[3];
    for (int q = 0; q < 3; ++q) nv[q] = (double*)malloc(sizeof(double) * (size_t)H);
    for (int64_t k = 0; k < M; ++k) {
        int n = (int)(leaves[k] >> 28);
        uint32_t i, j;
        orc_demorton(leaves[k] & 0x0FFFFFFFu, &i, &j);
        for (int q = 0; q < 3; ++q) nv[q][level_start(n) + rm(n, i, j)] = newU[3 * k + q];
    }
    for (int64_t sj = 0; sj < ns; ++sj)
        for (int64_t si = 0; si < ns; ++si) {
            int Ps = P[rm(Ls, si, sj)];
            int64_t w = side(Ps - Ls);
            for (int64_t jj = sj * w; jj < (sj + 1) * w; ++jj)
                for (int64_t ii = si * w; ii < (si + 1) * w; ++ii) {
                    int n = 0;                  /* the covering leaf (Algorithm 5's walk) */
                    while (n < Ps && S[level_start(n) + rm(n, ii >> (Ps - n), jj >> (Ps - n))]) n++;
                    int64_t kl = level_start(n) + rm(n, ii >> (Ps - n), jj >> (Ps - n));
                    int64_t kc = level_start(Ps) + rm(Ps, ii, jj);
                    double hl = nv[0][kl];
                    double hf = hl;
                    if (n < Ps && hl >= p->tol_h) {
                        double eta = hl + zh[kl];
                        double d = eta - zh[kc];
                        hf = d > 0.0 ? d : 0.0;
                    }
                    hier3[0][kc] = hf;
                    hier3[1][kc] = nv[1][kl];
                    hier3[2][kc] = nv[2][kl];
                }
        }
    for (int64_t s = 0; s < NSUB; ++s) m[s] = P[s];
    if (o) {
        if (o->T) memcpy(o->T, T, (size_t)P_);
        if (o->S) memcpy(o->S, S, (size_t)P_);
        if (o->leaves) memcpy(o->leaves, leaves, sizeof(uint32_t) * (size_t)(M < o->leaves_cap ? M : o->leaves_cap));
        o->num_leaves = M;
        o->dt_next = dt_from_rmin(p, rmin);
    }
    for (int q = 0; q < 3; ++q) { free(det[q]); free(nv[q]); }
    free(P); free(E); free(zh); free(zdet); free(T); free(S); free(leaves); free(newU);
    return 0;
}
