/*
 * oracle.h -- CPU FP64 oracle for the tetrahedral-FMM demagnetisation potential.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The CUDA
 * product path shares no code with it and never calls it.
 *
 * What it computes (Palmesi et al., Sec. 1, Eq. (1)-(2)):
 *     u(r) = 1/(4 pi) sum_j  int_{Omega_j} M_j(r') . grad'(1/|r - r'|) dr'
 * for tetrahedra Omega_j carrying an affine (P1, nodal) magnetisation M_j, with
 * u evaluated at the mesh nodes, and the mass-lumped field H = -grad u
 * (Sec. 4.1, "mass lumping was used for the computation of the B-field").
 *
 * Two evaluation routes:
 *   - oracle_direct:   the plain O(N_nodes * N_tets) definition, each tet
 *                      integrated in closed form (surface + volume charges);
 *   - oracle_fmm_eval: the method of Sec. 2-3 step by step: octree (Sec. 3.1),
 *                      radii + MAC (Sec. 3.2), dual tree traversal (Sec. 3.3,
 *                      Listings 1-2), exact tet moments (Sec. 2.2, Eq. expCoeffs),
 *                      M2M / M2L / L2L / L2P (Sec. 2 steps 2-5, Sec. 2.3) and
 *                      analytic P2P (Sec. 2.1).
 * Conventions: nodes are (N_n, 3) row-major doubles, tets (N_t, 4) 0-based
 * int32, M is (B, N_n, 3), u is (B, N_n), H is (B, N_n, 3).  Lengths in mesh
 * units, M in A/m, u in A, H in A/m; no mu0.
 */
#ifndef DEMAG_ORACLE_H
#define DEMAG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- single tetrahedron ------------------------------------------------ */
/* int_tet M(r').grad'(1/|r-r'|) dV' (no 1/4pi), M affine with nodal values
 * M[4][3] at the vertices v[4][3].  Closed form via surface and volume
 * charges; see oracle_direct.c for the derivation. */
double oracle_tet_potential(const double r[3], const double v[12], const double M[12]);
/* Same integral by the target-apex cone decomposition of Sec. 2.1 (Fig. 2)
 * with adaptive numerical quadrature over each face (the paper's own check of
 * its near field, Sec. 4).  rel_tol is the requested relative accuracy. */
double oracle_tet_potential_cone_quad(const double r[3], const double v[12], const double M[12],
                                      double rel_tol);
/* Same integral by a plain q^3-point collapsed Gauss-Legendre product rule over
 * the tet (only accurate for targets well away from the tet). */
double oracle_tet_potential_gauss3d(const double r[3], const double v[12], const double M[12], int q);

/* ---- whole mesh ------------------------------------------------------------ */
/* u[b*n_targets + i] for target nodes targets[i] (all nodes when targets==NULL,
 * then n_targets must equal n_nodes).  nthreads<=0: all cores. */
int oracle_direct(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                  const double* M, int B, const int64_t* targets, int64_t n_targets,
                  double* u, int nthreads);
/* Mass-lumped H (Sec. 4.1): H_i = -sum_{t ni i}|t| grad u_h|_t / sum_{t ni i}|t|. */
int oracle_lumped_H(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                    const double* u, int B, double* H);
/* Signed volumes (for the mesh-quality checks of the tests). */
/* The same u by the whole-mesh charge route: boundary-face surface charges
 * (bfaces: n_bfaces (tet, local face) pairs, face f opposite vertex f) plus the
 * volume charges of all tets; interior face charges cancel for continuous M. */
int oracle_direct_charges(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                          const int32_t* bfaces, int64_t n_bfaces, const double* M, int B,
                          const int64_t* targets, int64_t n_targets, double* u, int nthreads);
/* Pointwise H = -grad u at points off the boundary faces (whole-mesh charge
 * route, closed forms): H is B x n_pts x 3. */
int oracle_field_charges(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                         const int32_t* bfaces, int64_t n_bfaces, const double* M, int B, const double* pts,
                         int64_t n_pts, double* H, int nthreads);
void oracle_tet_volumes(const double* nodes, const int32_t* tets, int64_t n_tets, double* vol);

/* ---- expansions (Sec. 2.2-2.3) -------------------------------------------- */
/* Multi-indices |n|<=p in graded order: t=0..p, nx=t..0, ny=t-nx..0, nz=t-nx-ny. */
int  oracle_ncoef(int p);
void oracle_multi_indices(int p, int32_t* nxyz /* ncoef x 3 */);
/* D_n(x) = d^n (1/|x|) for all |n|<=p. */
void oracle_laplace_derivs(const double x[3], int p, double* D);
/* Exact moments Q_n = int_tet M.grad(y^n) dV, y = r' - c (Eq. expCoeffs), by a
 * collapsed Gauss-Legendre product rule exact for degree p. */
void oracle_tet_moments(const double v[12], const double M[12], const double c[3], int p, double* Q);
/* int_tet lambda_k y^m dV by the closed-form barycentric monomial integral
 * (multinomial expansion); independent check of the rule above. */
double oracle_tet_lambda_monomial_exact(const double v[12], const double c[3], int k,
                                        int mx, int my, int mz);
/* Translation operators, all on arrays of oracle_ncoef(p) doubles.
 *   M2M: Q^P_n = sum_{k<=n} C(n,k) d^{n-k} Q^C_k,           d = c_child - c_parent
 *   M2L: L_m  = 1/(4pi) sum_{|n|<=p-|m|} (-1)^|n|/n! D_{n+m}(R) Q_n,  R = c_T - c_S
 *   L2L: L^C_m = sum_{k>=m} L^P_k d^{k-m}/(k-m)!,           d = c_child - c_parent
 *   L2P: u(c+z) = sum_m L_m z^m/m!                                             */
void   oracle_m2m(int p, const double d[3], const double* Qc, double* Qp /* accumulated */);
void   oracle_m2l(int p, const double R[3], const double* Q, double* L /* accumulated */);
void   oracle_l2l(int p, const double d[3], const double* Lp, double* Lc /* accumulated */);
double oracle_l2p(int p, const double z[3], const double* L);
/* Far-field potential of a moment set about c: 1/(4pi) sum_n (-1)^|n|/n! D_n(r-c) Q_n. */
double oracle_multipole_eval(int p, const double c[3], const double* Q, const double r[3]);

/* ---- octree, radii, lists (Sec. 3.1-3.3) ---------------------------------- */
typedef struct oracle_tree oracle_tree;
/* status: 0 ok, 1 invalid argument. */
oracle_tree* oracle_tree_build(const double* nodes, int64_t n_nodes, const int32_t* tets,
                               int64_t n_tets, int leaf_size, double theta, int* status);
/* The same with the source model chosen: sources = 0, the tets binned by centroid
 * (the method); 1, point dipoles V_i M_i at the nodes (V_i the lumped volume),
 * with the node radius as source radius, point-dipole moments and near field
 * (self term left out); 2, vertex patches: node i carries lambda_i M_i over the
 * tets around it (the paper's hat-function clustering), binned by the node,
 * source radius the farthest vertex of those tets, exact moments and near field. */
oracle_tree* oracle_tree_build_sources(const double* nodes, int64_t n_nodes, const int32_t* tets,
                                       int64_t n_tets, int leaf_size, double theta, int sources, int* status);
void oracle_tree_free(oracle_tree* t);
/* info[0]=n_cells info[1]=n_m2l info[2]=n_p2p info[3]=n_levels info[4]=n_leaves */
void oracle_tree_info(const oracle_tree* t, int64_t* info);
/* Box: lo[3], side, scale. */
void oracle_tree_box(const oracle_tree* t, double* lo_side_scale);
/* Any pointer may be NULL.  Arrays sized by oracle_tree_info. */
void oracle_tree_export(const oracle_tree* t,
                        uint64_t* node_key, uint64_t* tet_key,      /* original order   */
                        int64_t* node_perm, int64_t* tet_perm,      /* sorted -> original */
                        int32_t* cell_level, uint64_t* cell_prefix,
                        int64_t* cell_ranges /* ncells x 4: tet_begin,tet_end,node_begin,node_end */,
                        int64_t* cell_parent, int64_t* cell_child /* ncells x 2: first, count */,
                        double* cell_centre /* ncells x 3 */, double* cell_radius /* ncells x 2: src,tgt */,
                        int64_t* m2l_off /* ncells+1 */, int64_t* m2l_src,
                        int64_t* p2p_off /* ncells+1 */, int64_t* p2p_src);

/* ---- FMM evaluation (Sec. 2 steps 1-5 + P2P) ------------------------------ */
/* u (B x n_nodes, original node order).  If target_leaves != NULL only the
 * nodes of those leaf cells are evaluated (others left untouched); the upward
 * pass is always complete.  nthreads<=0: all cores. */
int oracle_fmm_eval(const oracle_tree* t, int p, const double* M, int B, double* u,
                    const int64_t* target_leaves, int64_t n_target_leaves, int nthreads);

int oracle_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
