/*
 * masw_oracle.h -- declarations of the CPU FP64 oracle (test infrastructure
 * only; see masw_oracle.c for what each function follows in the paper).
 */
#ifndef MASW_ORACLE_H
#define MASW_ORACLE_H

#include <stdint.h>

#define ORACLE_OK 0
#define ORACLE_NO_ROOT 1
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)
#define ORACLE_MAX_LAYERS 256
#define ORACLE_MAX_KH 300.0

#ifdef __cplusplus
extern "C" {
#endif

double oracle_grid_velocity(double c0, double dc, int n);
void oracle_layer_stiffness(double k, double c, double h, double alpha, double beta,
                            double rho, double* Ke);
void oracle_halfspace_stiffness(double k, double c, double alpha, double beta, double rho,
                                double* Kh);
void oracle_assemble(int N, const double* h, const double* alpha, const double* beta,
                     const double* rho, double k, double c, double* K);
void oracle_lu_det(int n, double* A, int* sign, double* log_abs);
int oracle_det(int N, const double* h, const double* alpha, const double* beta,
               const double* rho, double k, double c, int* sign, double* log_abs);
int oracle_scan_limit(double beta_hs, double c0, double dc, int n_c);
int oracle_scan(int N, const double* h, const double* alpha, const double* beta,
                const double* rho, double lambda, double c0, double dc, int n_c, double* ct,
                int* idx);
int oracle_scan_changes(int N, const double* h, const double* alpha, const double* beta,
                        const double* rho, double lambda, double c0, double dc, int n_c,
                        int max_changes, int* idx, int* n_found);
int oracle_dispersion(int n_models, const int* n_layers, const double* h, const double* alpha,
                      const double* beta, const double* rho, const int* n_lambda,
                      const double* lambda, double c0, double dc, int n_c, double* ct,
                      int* idx, int* status, int n_threads);
int oracle_refine(int N, const double* h, const double* alpha, const double* beta,
                  const double* rho, double lambda, double c_lo, double c_hi, double rel_tol,
                  double* root);
int oracle_root(int N, const double* h, const double* alpha, const double* beta,
                const double* rho, double lambda, double c0, double dc, int n_c, int idx,
                double rel_tol, double* root);
int oracle_root_grad_fd(int N, const double* h, const double* alpha, const double* beta,
                        const double* rho, double lambda, double c0, double dc, int n_c,
                        int idx, double rel_step, double rel_tol, double* dC_dbeta,
                        double* dC_dh);
int oracle_det_leaky(int N, const double* h, const double* alpha, const double* beta,
                     const double* rho, double k, double c, int* sign_re, double* log_abs);
int oracle_scan_leaky(int N, const double* h, const double* alpha, const double* beta,
                      const double* rho, double lambda, double c0, double dc, int n_c,
                      double* ct, int* idx);
/* complex matrices as interleaved (re, im) doubles (C99 double complex) */
void oracle_halfspace_stiffness_complex(double k, double c, double alpha, double beta,
                                        double rho, double _Complex* Kh);
void oracle_assemble_complex(int N, const double* h, const double* alpha, const double* beta,
                             const double* rho, double k, double c, double _Complex* K);
void oracle_lu_det_complex(int n, double _Complex* A, double _Complex* phase, double* log_abs);
/* CPU banded baseline (the benchmark's second CPU line; pinned to the dense LU) */
int oracle_det_sign_banded(int N, const double* h, const double* alpha, const double* beta,
                           const double* rho, double k, double c, int* sign);
int oracle_scan_banded(int N, const double* h, const double* alpha, const double* beta,
                       const double* rho, double lambda, double c0, double dc, int n_c,
                       double* ct, int* idx);
int oracle_dispersion_banded(int n_models, const int* n_layers, const double* h,
                             const double* alpha, const double* beta, const double* rho,
                             const int* n_lambda, const double* lambda, double c0, double dc,
                             int n_c, double* ct, int* idx, int* status, int n_threads);
double oracle_misfit_paper(int L, const double* ct, const double* ce);
double oracle_misfit_lsq(int L, const double* ct, const double* ce, double sigma);

#ifdef __cplusplus
}
#endif
#endif
