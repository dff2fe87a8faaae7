/*
 * fmm_oracle.h -- plain FP64 CPU oracle for the 3D Laplace (1/r) FMM mat-vec.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The GPU library
 * shares no code, header, table or constant with it.
 *
 * What it computes (Yokota, Ibeid & Keyes, "Fast Multipole Method as a
 * Matrix-Free Hierarchical Low-Rank Approximation"):
 *   - the O(N^2) direct sum phi_i = sum_{j != i} q_j / |x_i - x_j| and its
 *     gradient g_i = grad phi(x_i) (the dense diagonal blocks of the
 *     hierarchical matrix are exactly this Green's-function operator, §2.2);
 *   - the analytic FMM (Greengard & Rokhlin, cited in §2.1) as a matrix-free
 *     H^2 mat-vec (§1, §2.4): octree over a Morton (3D->1D) ordering (§3.1),
 *     interaction list "children of the parent's neighbours that are not
 *     neighbours", at most 6^3 - 3^3 = 189 boxes (§2.2), and the adaptive
 *     U/W/X lists of the kernel-independent FMM paper the review cites
 *     (Ying, Biros & Zorin 2004).
 *
 * The paper prints no expansion formula.  The oracle uses complex solid
 * harmonics with Condon-Shortley phase and the normalisation
 *     R_n^m(x) = r^n P_n^m(cos t) e^{i m p} / (n+m)!      (regular)
 *     I_n^m(x) = (n-m)! P_n^m(cos t) e^{i m p} / r^{n+1}  (irregular)
 *     R_n^{-m} = (-1)^m conj(R_n^m),  I_n^{-m} = (-1)^m conj(I_n^m),
 * for which the addition theorem takes the coefficient-free forms
 *     R_n^m(a+b)   = sum_{k,l} R_k^l(a) R_{n-k}^{m-l}(b)
 *     1/|x-y|      = sum_{n,m} conj(R_n^m(y)) I_n^m(x),             |y|<|x|
 *     I_k^l(d+u)   = sum_{n,m} (-1)^n conj(R_n^m(u)) I_{n+k}^{m+l}(d), |u|<|d|
 * Every translation below is one of these identities truncated at degree p;
 * each is pinned by the tests against direct sums.
 *
 * Complex coefficient arrays hold (p+1)^2 entries, index n*n+n+m for
 * -n <= m <= n, stored as interleaved (re, im) doubles.
 */
#ifndef FMM_ORACLE_H
#define FMM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- solid harmonics (pinned against the associated Legendre functions) */
void oracle_regular(int p, const double x[3], double *R);   /* (p+1)^2 complex */
void oracle_irregular(int p, const double x[3], double *I); /* (p+1)^2 complex */

/* ---- direct sum: targets vs all sources, pairs at zero distance skipped.
 *      grad may be NULL.  phi[nt], grad[3*nt] are overwritten. */
void oracle_direct(int64_t ns, const double *src_xyz, const double *q,
                   int64_t nt, const double *tgt_xyz, double *phi, double *grad);

/* ---- single translations about explicit centres (absolute coordinates).
 *      All accumulate (+=) into their output. */
void oracle_p2m(int p, const double c[3], int64_t n, const double *xyz,
                const double *q, double *M);
void oracle_m2m(int p, const double c_child[3], const double *Mc,
                const double c_parent[3], double *Mp);
void oracle_m2l(int p, const double c_src[3], const double *M,
                const double c_tgt[3], double *L);
void oracle_l2l(int p, const double c_parent[3], const double *Lp,
                const double c_child[3], double *Lc);
void oracle_p2l(int p, const double c[3], int64_t n, const double *xyz,
                const double *q, double *L);
/* evaluation: phi[n] and grad[3n] accumulate; grad may be NULL */
void oracle_l2p(int p, const double c[3], const double *L, int64_t n,
                const double *xyz, double *phi, double *grad);
void oracle_m2p(int p, const double c[3], const double *M, int64_t n,
                const double *xyz, double *phi, double *grad);

/* ---- root cube and Morton keys (§3.1).
 *   lo = per-axis minimum; D = smallest power of two strictly above the
 *   largest per-axis extent (1 if all points coincide);
 *   q_a = min(floor((x_a - lo_a) * 2^21 / D), 2^21 - 1);
 *   key bit 3b+0 = bit b of q_x, 3b+1 = bit b of q_y, 3b+2 = bit b of q_z.
 *   Returns 0, or -1 when a coordinate is not finite. */
int oracle_root_cube(int64_t n, const double *xyz, double lo[3], double *D);
void oracle_morton_keys(int64_t n, const double *xyz, const double lo[3],
                        double D, uint64_t *keys);

/* ---- adaptive octree + interaction lists.
 * Boxes are numbered by (level, Morton key) ascending.  A box at level
 * l < max_depth holding more than leaf_size points splits into its
 * non-empty octants. */
typedef struct oracle_tree oracle_tree;
oracle_tree *oracle_tree_build(int64_t n, const double *xyz, int leaf_size,
                               int max_depth);
void oracle_tree_free(oracle_tree *t);
/* Move every W pair of two leaves (B, A in W(B)) whose W leaf A holds at most
 * max_points points to the near field in both directions: A joins U(B), B
 * joins U(A); A leaves W(B), B leaves X(A).  Rows stay sorted. */
void oracle_tree_direct_wx(oracle_tree *t, int max_points);

/* sizes: [0]=n [1]=nboxes [2]=nlevels [3]=|U| [4]=|V| [5]=|W| [6]=|X| */
void oracle_tree_sizes(const oracle_tree *t, int64_t sizes[7]);
void oracle_tree_geometry(const oracle_tree *t, double lo[3], double *D);
/* Any pointer may be NULL (that array is skipped).  Sizes from
 * oracle_tree_sizes: keys/perm n; level_offset nlevels+1; box_* nboxes;
 * *_off nboxes+1; *_idx the list sizes. */
void oracle_tree_export(const oracle_tree *t, uint64_t *keys, int32_t *perm,
                        int32_t *level_offset, uint64_t *box_key,
                        int32_t *box_level, int32_t *box_first,
                        int32_t *box_count, int32_t *box_parent,
                        int32_t *box_child, int32_t *box_nchild,
                        int32_t *u_off, int32_t *u_idx, int32_t *v_off,
                        int32_t *v_idx, int32_t *w_off, int32_t *w_idx,
                        int32_t *x_off, int32_t *x_idx);

/* ---- FMM mat-vec with order p on a built tree.  q, phi, grad in the
 *      caller's (input) order; grad may be NULL. */
void oracle_fmm_eval(const oracle_tree *t, int p, const double *q,
                     double *phi, double *grad);

/* ---- dual-tree traversal with a multipole acceptance criterion (§2.1):
 * cell radius r_B = max |x_j - c_B| over B's points; (T, S) accepted for M2L
 * iff r_T + r_S < theta |c_T - c_S|; rejected pairs split symmetrically
 * (both leaves -> P2P; one leaf -> the other; coarser cell; same level ->
 * both).  Lists per target box, sources ascending. */
typedef struct oracle_dual oracle_dual;
oracle_dual *oracle_dual_build(const oracle_tree *t, double theta);
void oracle_dual_free(oracle_dual *d);
/* sizes: [0] = M2L pairs, [1] = P2P leaf pairs */
void oracle_dual_sizes(const oracle_dual *d, int64_t sizes[2]);
/* offsets nboxes+1, sources, radius nboxes; any pointer may be NULL */
void oracle_dual_export(const oracle_dual *d, int32_t *m2l_off, int32_t *m2l_idx,
                        int32_t *p2p_off, int32_t *p2p_idx, double *radius);
/* FMM mat-vec over the dual-tree lists (M2M to the root, M2L over the
 * accepted pairs, L2L from the root, L2P + P2P at the leaves) */
void oracle_dual_eval(const oracle_tree *t, const oracle_dual *d, int p, const double *q,
                      double *phi, double *grad);

/* ---- Helmholtz kernel e^{i kappa r}/r (helmholtz_oracle.c; basis and
 *      translation identities in that file's preamble).  Complex arrays are
 *      interleaved (re, im); coefficient index n*n+n+m. */
void oracle_sph_bessel(int nmax, double x, double *j, double *y); /* y may be NULL */
void oracle_sph_harmonics(int p, const double x[3], double *Y);  /* (p+1)^2 complex */
void oracle_h_wave(int p, double kappa, const double x[3], int singular, double *X);
void oracle_gauss_legendre(int n, double *x, double *w);
int64_t oracle_gaunt_size(int p);
void oracle_gaunt_table(int p, double *G);
void oracle_h_translate(int p, double kappa, const double *G, const double t[3], int singular,
                        const double *in, double *out);
void oracle_h_direct(int64_t ns, const double *src, const double *q, int64_t nt,
                     const double *tgt, double kappa, double *phi);
void oracle_h_p2m(int p, double kappa, const double c[3], int64_t n, const double *xyz,
                  const double *q, double *M);
void oracle_h_p2l(int p, double kappa, const double c[3], int64_t n, const double *xyz,
                  const double *q, double *L);
void oracle_h_m2m(int p, double kappa, const double *G, const double c_child[3],
                  const double *Mc, const double c_parent[3], double *Mp);
void oracle_h_m2l(int p, double kappa, const double *G, const double c_src[3], const double *M,
                  const double c_tgt[3], double *L);
void oracle_h_l2l(int p, double kappa, const double *G, const double c_parent[3],
                  const double *Lp, const double c_child[3], double *Lc);
void oracle_h_l2p(int p, double kappa, const double c[3], const double *L, int64_t n,
                  const double *xyz, double *phi);
void oracle_h_m2p(int p, double kappa, const double c[3], const double *M, int64_t n,
                  const double *xyz, double *phi);
void oracle_h_fmm_eval(const oracle_tree *t, int p, double kappa, const double *q,
                       double *phi);

/* number of OpenMP threads the oracle runs with (1 without OpenMP) */
int oracle_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
