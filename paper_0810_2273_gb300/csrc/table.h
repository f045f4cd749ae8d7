// Host-side kernel-table construction (internal to libvdwdf).
#pragma once

namespace vdwdf {

// phi at the nodes D_k = Dmax k/(nD-1), delta_l = l/ndelta by quadrature of
// Dion eq. (14); row k = 0 softened (see table.cpp).  nodes: nD*ndelta, D outer.
// level: 0 fast, 1 standard, 2 fine.  Returns 0 or -1 on allocation failure.
int build_phi_nodes(int nD, double Dmax, int ndelta, int level, double *nodes);

// Number of quadrature nodes per axis at a level.
int quadrature_node_count(int level);

// Bicubic B-spline coefficients (nD + 2) x (ndelta + 2), D outer, of the
// tensor-product cubic spline through nodes with zero slope at D = 0 and
// delta = 0 and zero curvature at the last node of each axis.
void spline_coefficients(int nD, int ndelta, const double *nodes, double *coef);

// 1-D cubic B-spline coefficients (ndelta + 2) in delta of
// rho(delta_l) = phi(Dmax, delta_l) / phi17(Dmax, delta_l) (same end conditions),
// which scales Dion's eq. (17) beyond the table so that phi is continuous at Dmax.
void rho_coefficients(int nD, double Dmax, int ndelta, const double *nodes, double *coef);

}  // namespace vdwdf
