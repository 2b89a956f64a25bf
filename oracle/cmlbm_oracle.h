/*
 * cmlbm_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow FP64 CPU restatement of the D3Q27 central-moment lattice Boltzmann
 * scheme with external forcing of De Rosis, Huang & Coreixas (arXiv 1905.10182).
 * It exists to check the CUDA path.  Only the test suite, the smoke entry point and
 * the benchmark's CPU-baseline leg may load it; the product library never does.
 * It shares no code, header, table or constant with the CUDA path.
 *
 * Conventions
 *   - Population i of node n = x + nx*(y + ny*z) is f[i*N + n], N = nx*ny*nz
 *     (structure of arrays, x fastest), values are full populations f_i (not
 *     deviations), FP64.
 *   - Lattice units; c_s^2 = 1/3 (Sec. II, below Eq. eq:truncation).
 *   - Force F is a force density: the forcing term carries no rho prefactor
 *     (reading of Eq. forcing that reproduces Eq. force_cms_sixth and Eq. macroscopic).
 */
#ifndef CMLBM_ORACLE_H
#define CMLBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_Q 27

/* collision operators */
enum {
    ORC_COLL_LITERAL = 0, /* k* = (I-L)T^T f + L T^T feq + (I-L/2) T^T F, f* = (T^T)^-1 k*   (Sec. II) */
    ORC_COLL_PAPER   = 1, /* five-step summary of Sec. II: closed-form post-collision CMs + fast CM inverse */
    ORC_COLL_BGK     = 2, /* single-rate BGK, Eq. collision */
    ORC_COLL_NONE    = 3  /* identity: pure streaming, used to label populations and check indices */
};

/* force sources */
enum {
    ORC_FORCE_NONE = 0,
    ORC_FORCE_UNIFORM = 1,    /* F = (force[0], force[1], force[2]) everywhere                   */
    ORC_FORCE_KOLMOGOROV = 2, /* F_x = force[0] * sin(2 pi y / ny), F_y = F_z = 0                */
    ORC_FORCE_FIELD = 3,      /* F from fx, fy, fz arrays (N each)                               */
    ORC_FORCE_SHAN_CHEN = 4   /* F = -G psi(x) sum_i w_i c_i psi(x + c_i), psi = 1 - exp(-rho)  (Sec. III, static droplet) */
};

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_SINGULAR = 2, ORC_ERR_NOMEM = 3 };

typedef struct {
    int nx, ny, nz;
    double omega;               /* rate of the second-order moments k4..k8, Eq. eq:relaxationMatrix */
    double rho0;                /* reference density, used only by orc_init_rest */
    int walls_y;                /* 1: halfway bounce-back walls at y = -1/2 and y = ny - 1/2 */
    const unsigned char* mask;  /* NULL or N bytes, 1 = solid node */
    int collision;              /* ORC_COLL_* */
    int eq_order;               /* Hermite order kept in feq   (LITERAL only; 6 = complete, Eq. eq:truncation) */
    int force_order;            /* Hermite order kept in F_i   (LITERAL only; 6 = complete, Eq. forcing)       */
    const double* lambda;       /* LITERAL/BGK override: 27 relaxation rates, NULL = paper's Lambda */
    int force_kind;             /* ORC_FORCE_* */
    double force[3];
    double G;                   /* Shan-Chen interaction strength */
    const double* fx;
    const double* fy;
    const double* fz;
    int threads;                /* OpenMP threads, <= 0 = runtime default */
} orc_desc;

/* lattice (Sec. II): velocities in the paper's order, weights, opposite direction */
void orc_velocities(int c[ORC_Q * 3]);
void orc_weights(double w[ORC_Q]);
int orc_opposite(int i);

/* Hermite tensor H_{nx ny nz}(c_i) of App. A (tensor product of 1D polynomials) */
double orc_hermite(int i, int nx, int ny, int nz);

/* Eq. eq:truncation, keeping Hermite tensors of total order <= order (6 = complete) */
void orc_equilibrium(double rho, const double u[3], int order, double feq[ORC_Q]);
/* Eq. forcing / Eq. generalForcing, keeping Hermite tensors of total order <= order (6 = complete) */
void orc_forcing_term(const double F[3], const double u[3], int order, double Fi[ORC_Q]);
/* Eq. basis: T[i*27 + j] = T_j evaluated at the shifted velocity c_i - u */
void orc_basis(const double u[3], double T[ORC_Q * ORC_Q]);
/* k = T^T v (central moments of any population-space vector) */
void orc_central_moments(const double u[3], const double v[ORC_Q], double k[ORC_Q]);
/* solve (T^T) v = k for v: the literal inverse of Eq. system */
int orc_inverse_literal(const double u[3], const double k[ORC_Q], double v[ORC_Q]);
/* the same inverse through the fast CM transform (three 1D D1Q3 inverses) */
void orc_inverse_fast(const double u[3], const double k[ORC_Q], double v[ORC_Q]);

/* One node's collision; F is the force density at the node. */
int orc_collide(const orc_desc* d, const double f[ORC_Q], const double F[3], double fstar[ORC_Q]);

/* Macroscopic fields of Eq. macroscopic (u includes F/2). rho: N, u: 3N (ux block, uy, uz). */
int orc_force_field(const orc_desc* d, const double* f, double* F3);
int orc_macroscopic(const orc_desc* d, const double* f, double* rho, double* u3);

/* f = feq(rho, u) (complete equilibrium) on every fluid node; solid nodes get feq(rho0, 0). */
int orc_init_equilibrium(const orc_desc* d, const double* rho, const double* u3, double* f);

/* nsteps of collide (Eq. collision / Sec. II) + two-array streaming (Eq. streaming) with
   halfway bounce-back at walls and solid nodes; f is updated in place. */
int orc_step(const orc_desc* d, double* f, int nsteps);

/* One step evaluated only at the listed nodes: out[k*27 + i] = f_i(nodes[k], t+1). */
int orc_step_sampled(const orc_desc* d, const double* f, const long long* nodes, int count, double* out);

/* ------------------------------------------------------------------ magnetic field (App. C)
 * A second LBM on D3Q7 for the magnetic field b: vector populations h_l (l = 0..6, velocities
 * xi_l = 0, +-x, +-y, +-z), stored h[(3*l + a)*N + n] (component a = x, y, z of population l),
 * BGK with omega_m, eta = cs_m^2 (1/omega_m - 1/2), cs_m^2 = 1/4, weights 1/4 and 1/8,
 *   h_la^eq = w_l [ b_a + 4 xi_lb (u_b b_a - b_b u_a) ],    b = sum_l h_l.
 * Coupling (readings): the Lorentz force F_L = j x b is added to the fluid's force density; the
 * current j = curl b comes from the non-equilibrium electric tensor of the pre-collision h,
 * d_b b_a = -(omega_m / cs_m^2) sum_l xi_lb (h_la - h_la^eq), i.e. j = -(omega_m / cs_m^2)(E - 2 u x b)
 * with E_g = eps_gba sum_l xi_lb h_la; u (which both h^eq and Eq. macroscopic use) and F_L are
 * solved together, rho u = sum_i f_i c_i + (F_ext + F_L)/2, which is linear in u.  Walls: halfway
 * (y = -1/2, ny - 1/2) anti-bounce-back h_l(x, t+1) = -h*_opp(l)(x, t) + 2 w_l b_wall, which holds
 * b = b_wall on the wall to second order. */
#define ORC_QM 7
void orc_mhd_velocities(int xi[ORC_QM * 3]);
void orc_mhd_weights(double w[ORC_QM]);
/* h_la^eq, heq[3*l + a] */
void orc_mhd_equilibrium(const double b[3], const double u[3], double heq[ORC_QM * 3]);
/* b = sum_l h_l and E_g = eps_gba sum_l xi_lb h_la of one node's populations h[3*l + a] */
void orc_mhd_moments(const double h[ORC_QM * 3], double b[3], double E[3]);
/* rho, u, Lorentz force and current of one node from its fluid populations (27, full f), its
 * magnetic populations and the external force density */
void orc_mhd_node(const double f[ORC_Q], const double h[ORC_QM * 3], const double Fext[3], double omega_m,
                  double* rho, double u[3], double FL[3], double j[3]);
/* h = h^eq(b, u) on every node; b3, u3: 3N arrays (x block, y, z) */
int orc_mhd_init(const orc_desc* d, const double* b3, const double* u3, double* h);
/* nsteps of the coupled scheme: fluid collision (d->collision, force = F_ext + F_L; F_ext from
 * d->force_kind NONE or UNIFORM), magnetic BGK, two-array streaming of both (fluid: halfway
 * bounce-back; magnetic: anti-bounce-back with b_wall).  No masks. */
int orc_mhd_step(const orc_desc* d, double omega_m, const double b_wall[3], double* f, double* h, int nsteps);
/* rho (N), u, b, j (3N each) at the current time */
int orc_mhd_fields(const orc_desc* d, double omega_m, const double* f, const double* h, double* rho, double* u3,
                   double* b3, double* j3);

/* ------------------------------------------------------------------ colour gradient (App. D)
 * Two immiscible fluids, red and blue, with D3Q27 populations fr, fb (full populations, layout of
 * f); the total f = fr + fb takes the central-moment collision of Sec. II with an enhanced
 * equilibrium, then a perturbation (interfacial tension) and a recolouring step split it again.
 * Per node (readings where App. D is silent or garbled):
 *   rho_k = sum fk, rho = rho_r + rho_b, rho u = sum f c + F/2,
 *   phi = (rho_r/rho_r0 - rho_b/rho_b0) / (rho_r/rho_r0 + rho_b/rho_b0),
 *   alpha_b = 8/27, alpha_r = 1 - (1 - alpha_b) rho_b0 / rho_r0, alpha = ((1+phi) alpha_r + (1-phi) alpha_b)/2,
 *   1/nu = (1+phi)/(2 nu_r) + (1-phi)/(2 nu_b), omega = 1/(3 nu + 1/2) on k4..k8;
 *   gradients grad X = (1/cs^2) sum_i w_i c_i X(x + c_i), a missing neighbour behind a wall
 *   taking the node's own value;
 *   f^eq_i = rho phi_i(alpha) + (f^eq,complete_i(rho, u) - rho w_i) + Phi_i (the enhanced
 *   equilibrium of App. D: the sixth-order Hermite terms of Eq. eq:truncation without their
 *   zeroth-order term), Phi_i from G = (u grad rho + grad rho u) / 48;
 *   single phase: k* = (I - L) k + L k^eq + (I - L/2) R, f* = (T^T)^-1 k* (R: the complete
 *   forcing term of Eq. generalForcing);
 *   perturbation: f* += (A/2)|grad phi| [w_i (c_i . grad phi)^2 / |grad phi|^2 - B_i] (squared, so
 *   that it conserves mass);
 *   recolouring: fr*_i = (rho_r/rho) f*_i + beta rho_r rho_b / rho^2 cos(theta_i) rho phi_i(alpha),
 *   fb*_i = f*_i - fr*_i, cos(theta_i) = c_i . grad phi / (|c_i| |grad phi|);
 *   body force (Sec. III, Rayleigh-Taylor): F = (rho - (rho_r0 + rho_b0)/2) gvec. */
typedef struct {
    const orc_desc* grid;  /* nx, ny, nz, walls_y, threads (collision, force and mask fields unused) */
    double rho_r0, rho_b0; /* reference densities of the pure fluids */
    double nu_r, nu_b;
    double A;              /* perturbation amplitude */
    double beta;           /* recolouring parameter */
    double gvec[3];        /* gravity vector of the body force */
} orc_cg;
/* phi_i(alpha) of App. D */
void orc_cg_phi(double alpha, double phi_i[ORC_Q]);
/* enhanced equilibrium */
void orc_cg_equilibrium(double rho, const double u[3], double alpha, double nu, const double grad_rho[3],
                        double feq[ORC_Q]);
/* perturbation operator values */
void orc_cg_perturbation(double A, const double grad_phi[3], double out[ORC_Q]);
/* recolouring of the post-collision total fs into fr, fb */
void orc_cg_recolour(double beta, double rho_r, double rho_b, double alpha, const double grad_phi[3],
                     const double fs[ORC_Q], double fr[ORC_Q], double fb[ORC_Q]);
/* initial state: fk_i = (rho_k / rho) f^eq_i(rho, u) with the enhanced equilibrium at alpha(phi)
   and no density-gradient term */
int orc_cg_init(const orc_cg* m, const double* rho_r, const double* rho_b, const double* u3, double* fr, double* fb);
int orc_cg_step(const orc_cg* m, double* fr, double* fb, int nsteps);
/* rho_r, rho_b (N each), u (3N) */
int orc_cg_fields(const orc_cg* m, const double* fr, const double* fb, double* rho_r, double* rho_b, double* u3);

#ifdef __cplusplus
}
#endif
#endif
