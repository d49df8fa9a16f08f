/*
 * clbm_oracle.h -- FP64 CPU oracle of the D3Q19 cascaded central-moment lattice
 * Boltzmann method for power-law fluids (Adam, Hajabdollahi & Premnath,
 * "Cascaded lattice Boltzmann modeling and simulations of three-dimensional
 * non-Newtonian fluid flows", Sec. 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * includes this file.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code, table or header
 * with the CUDA path.
 *
 * Storage: plain (unshifted) populations f[q][z][y][x], x fastest, FP64.
 * The stored array always holds POST-collision populations; one step pulls
 * them along the lattice links (streaming, Eq. cascadedstreaming1) and
 * collides (Eq. cascadedcollision1).
 */
#ifndef CLBM_ORACLE_H
#define CLBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Face kinds, faces ordered (-x, +x, -y, +y, -z, +z). */
enum { ORC_PERIODIC = 0, ORC_WALL = 1, ORC_LID = 2 };

typedef struct {
  int nx, ny, nz;
  int face[6];
  double K;          /* consistency coefficient mu_p (Eq. 5) */
  double n;          /* power-law index (Eq. 5) */
  double U[3];       /* velocity of every LID face (must be tangential) */
  double F[3];       /* body force per unit volume */
  double rho0;       /* reference density: rest state and lid wall density */
  double nu_min;     /* kinematic viscosity clamp (reading: clamps) */
  double nu_max;
  double omega[19];  /* omega[9..18]: relaxation rates of bulk and higher
                        moments (Sec. 3.1 sets them to 1); 0..8 unused */
  int attractor_over_rho; /* 1: 4th-order attractor k~ii k~jj / rho (reading);
                             0: the literal printed product k~ii k~jj */
} orc_params;

/* Per-node diagnostics of one collision. */
typedef struct {
  double rho;
  double u[3];       /* u* = (j + F/2)/rho, the output velocity */
  double gamma_dot;  /* |gamma_dot| at the solved omega (Eq. shearrateexpression) */
  double omega_nu;   /* omega_4..omega_8 (Eq. localvarationsrelaxationtimes) */
  double g[19];      /* change of moments g^_0..g^_18 (g^_0..3 = 0) */
} orc_node_info;

/* Lattice constants as the oracle builds them (for the pin tests). */
void orc_velocities(int e_out[19][3]);
void orc_weights(double w_out[19]);
/* K[alpha][j], built from the basis definitions (Sec. 3, |K_0>..|K_18>). */
void orc_kmatrix(double K_out[19][19]);

/* Fill the parameter struct with the defaults (rho0 = 1, clamps 5e-4 / 10,
 * omega_9..18 = 1, attractor over rho, all faces periodic). */
void orc_default_params(orc_params* p);

/* Solve omega_nu from the non-equilibrium second moments m^(1)_4..9 (Eqs.
 * strainratetensor, localvarationsrelaxationtimes, 6) by bisection.
 * Returns omega, writes |gamma_dot| at that omega. */
double orc_omega_solve(const orc_params* p, double rho, const double m[10],
                       double* gamma_dot);

/* One collision of a single node: f (19, pre-collision, post-streaming) ->
 * ft (19, post-collision).  info may be NULL. */
void orc_collide(const orc_params* p, const double f[19], double ft[19],
                 orc_node_info* info);

/* State of rest: f = w rho0 everywhere.  f has 19*nx*ny*nz entries. */
void orc_rest_state(const orc_params* p, double* f);

/* nsteps full steps (pull-stream with boundaries, then collide).  A holds the
 * state on entry and on return; B is a work buffer of the same size. */
int orc_run(const orc_params* p, double* A, double* B, int64_t nsteps);

/* The streamed (pre-collision) populations of every node: out[q][z][y][x]. */
void orc_pull(const orc_params* p, const double* A, double* out);

/* Macroscopic fields of the current state: rho, u (3 x N, SoA: ux then uy
 * then uz) and |gamma_dot|, computed from the streamed populations.  Any
 * output pointer may be NULL. */
void orc_fields(const orc_params* p, const double* A, double* rho, double* u,
                double* gamma_dot);

/* Steady-state residual (reading: residual)
 *   R = ||u - u_prev||_2 / (delta * ||u||_2)   over N nodes, u as 3 x N. */
double orc_residual(const double* u, const double* u_prev, int64_t N,
                    int64_t delta);

/* Total mass sum(f) of a state. */
double orc_mass(const orc_params* p, const double* A);

#ifdef __cplusplus
}
#endif
#endif
