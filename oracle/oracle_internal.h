/* Internal helpers shared by the oracle's own C files (test infrastructure
 * only; never included by the CUDA library). */
#ifndef AETHER_ORACLE_INTERNAL_H
#define AETHER_ORACLE_INTERNAL_H

#include "oracle.h"

/* Ghosted mesh: every array spans indices -ng .. n+ng along each axis
 * (n + 2 ng + 1 points, so face arrays fit), i fastest. */
typedef struct {
  int n[3], ng, N[3];
  long size;
  int coord;
  double lo[3], hi[3], dx[3];
  int bc[3];
} Mesh;

#define IDX(m, i, j, k)                                                  \
  ((((long)(k) + (m)->ng) * (m)->N[1] + ((j) + (m)->ng)) * (m)->N[0] + \
   ((i) + (m)->ng))

int orc_mesh_init(Mesh* m, const orc_grid* g, int ng);
double orc_xf(const Mesh* m, int d, int i);
double orc_area(const Mesh* m, int d, int i, int j, int k);
double orc_volume(const Mesh* m, int i, int j, int k);
double orc_edge(const Mesh* m, int d, int i, int j, int k);
void orc_widths(const Mesh* m, int i, int j, int k, double* w);
void orc_fill_ghosts(const Mesh* m, double** u, int nu, double** b);
int orc_ghost_width(int recon);
void orc_load(const Mesh* m, const double* cons, const double* b1,
              const double* b2, const double* b3, double** u, int nu,
              double** b);
void orc_store(const Mesh* m, double** u, int nu, double** b, double* cons,
               double* b1, double* b2, double* b3);



/* Fast magnetosonic speed along the normal of a face-frame state, and the
 * conserved vector, physical flux and total pressure of one side (mhd.c). */
double orc_fast_speed(double gamma, double rho, double p, double bn, double bt1, double bt2);
void orc_side_flux(double gamma, const double* w, double bn, double* u, double* f, double* pt);

/* L(U) of Eq. 8 (gas, hydro or MHD) on the interior; see mhd.c. */
long orc_rhs(const Mesh* m, const orc_params* p, int recon, double** u, double** b,
             double** out_u, double** out_b);
#endif
