/*
 * FP64 CPU oracle of the collapse-time step (Sec. 2.1.1).  TEST
 * INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.
 *
 * Complex arrays are interleaved (re, im) doubles.  Half-spectra are
 * [n][n][n/2+1]; real fields and outputs are [n][n][n], q = (x n + y) n + z.
 * The *3 variants take a grid of nx x ny x nz points with cubic cells (box
 * is the side along x): half-spectra [nx][ny][nz/2+1], fields [nx][ny][nz].
 * Hessian components are ordered xx, yy, zz, xy, xz, yz.
 */
#ifndef PIN_ORACLE_H
#define PIN_ORACLE_H

void or_dft1d(const double* in_ri, int n, int sign, double* out_ri);
void or_idft3d(double* a_ri, int n);
int or_hessian(const double* delta_half_ri, int n, double box, double radius, double* out6,
               double* max_imag);
double or_hessian_point(const double* delta_half_ri, int n, double box, double radius,
                        int comp, int qx, int qy, int qz);
int or_hessian_points(const double* delta_half_ri, int n, double box, double radius, int npts,
                      const long long* q_list, double* out);
int or_displacement(const double* delta_half_ri, int n, double box, double* out3);
int or_displacement_r(const double* delta_half_ri, int n, double box, double radius, double* out3);
int or_hessian3(const double* delta_half_ri, int nx, int ny, int nz, double box, double radius,
                double* out6, double* max_imag);
int or_displacement3(const double* delta_half_ri, int nx, int ny, int nz, double box, double radius,
                     double* out3);
int or_collapse_times3(const double* delta_half_ri, int nx, int ny, int nz, double box, int nscales,
                       const double* radii, int correction, double* fmax, int* idx,
                       double* f_all, double* f2, int* idx2, double* slope, double* vmax,
                       double* hrms);
void or_eig3(const double* h6, double* lam);
void or_axis_coeffs(const double* lam, int i, double* c);
double or_first_root(const double* c);
double or_delta_c(void);
double or_x3(void);
double or_collapse_F(const double* lam, int correction);
double or_collapse_point(const double* h6, int correction, double* lam_out);
double or_collapse_slope(const double* lam);
int or_collapse_times(const double* delta_half_ri, int n, double box, int nscales,
                      const double* radii, int correction, double* fmax, int* idx,
                      double* f_all, double* f2, int* idx2, double* slope, double* vmax);
int or_collapse_times_sampled(const double* delta_half_ri, int n, double box, int nscales,
                              const double* radii, int correction, int npts,
                              const long long* q_list, double* fmax, int* idx, double* f2,
                              int* idx2);
void or_collapse_interval(const double* h6s, const double* hscale, int nscales, int npts, int correction,
                          double u, double* lo, double* hi);
void or_collapse_from_hessians(const double* h6s, int nscales, int npts, int correction,
                               double* fmax, int* idx, double* f2, int* idx2);

#endif
