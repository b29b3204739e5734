// Host-side construction of the univariate IFFD data (one parametric direction).
//
// Everything here runs once per (n, p, Dirichlet set) on the CPU in float64 and
// produces the small tables the CUDA passes consume. No device code.
#pragma once

#include <string>
#include <utility>
#include <vector>

namespace iffd {

// Transform families of Table 1 that the device passes implement.
enum TransformKind : int {
  TK_DST1 = 0,   // p odd, D = {0,1}: U_reg = DST-I, U_reg^T = DST-I
  TK_DST23 = 1,  // p even, D = {0,1}: U_reg = DST-III, U_reg^T = DST-II
  TK_GEN = 2,    // the other six cases of Table 1 (DST-III/IV, DCT-I..IV types):
                 // U_ij = sin(pi (i - c)(j - e) / n + beta) via a zero-padded DFT
};

struct Axis1D {
  int n = 0, p = 0;          // elements, degree
  bool dir0 = true, dir1 = true;  // Dirichlet data at x = 0 / x = 1
  // repeated interior breakpoints (k, e): z_k = k/n appears 1 + e times in the
  // knot vector (continuity C^{p-1-e} there; Remark "reduced_regularity")
  std::vector<std::pair<int, int>> reps;
  int m = 0;                 // dim S_{p,h,D} = n + p + sum e - |D|
  int n_reg = 0, n_out = 0;  // eq. "reg_space_dim"
  int kind = TK_DST23;
  // TK_GEN: DFT length 2 n gq; frequency of output j is gq j - gqe (FWD) and
  // of output i is gq i - gqc (BWD), i.e. q (j - e) and q (i - c).
  int gq = 1, gqc = 0, gqe = 0;
  // TK_GEN post factors: w_j / D~_j (2 n_reg, complex), v_i (2 n_reg, complex),
  // 1 / D~_j (n_reg)
  std::vector<double> gpost;
  // V_reg (Section 4): rows 0..rowsL-1 x cols 0..nL-1 is the left edge block,
  // the right edge block is the mirror image of VR: V_reg[m-1-r][n_reg-1-c] =
  // VR[r][c] (c < nR, r < rowsR). An interior special function j (nL <= j <
  // n_reg - nR) is either the B-spline with reduced index j + offset, where
  // the offset is o before the first interior block and blk[6b+4] after block
  // b, or a column of an interior block b: columns [blk[6b], blk[6b+1]) x rows
  // [blk[6b+2], blk[6b+3]), dense row-major at VB + blk[6b+5]. Interior blocks
  // exist only around repeated knots; blocks are ordered by columns and rows.
  int nL = 0, rowsL = 0, o = 0, nR = 0, rowsR = 0;
  std::vector<double> VL;    // rowsL * nL, row-major
  std::vector<double> VR;    // rowsR * nR, row-major (left-end form of the right block)
  std::vector<int> blk;      // 6 per interior block: c0, c1, r0, r1, offset after, VB offset
  std::vector<double> VB;
  // W = V_out Q_out (m x n_out, row-major), significant only on rows
  // [0, wlo) and [whi, m); the rows in between are below 1e-17 of max |W|.
  std::vector<double> W;
  int wlo = 0, whi = 0;
  int wlo_f = 0, whi_f = 0;  // the same for FP32 passes (rows below 1e-10 of max |W|)
  std::vector<double> lam;    // Lambda~ diagonal: Lambda_reg (n_reg) then Lambda_out (n_out)
  std::vector<double> dtilde; // D~_reg diagonal (n_reg)
  // Banded mass / stiffness of S_{p,h,D}: band[i*(2p+1) + (j-i+p)] = A[i][j].
  std::vector<double> Mband, Kband;
  // Same, weighted by s(x) = sin(2 pi x) under the integral (variable
  // coefficient a = 1 + c prod_k s(x_k)); filled by build_weighted_bands.
  std::vector<double> Msband, Ksband;
};

// M^s_ij = int s B_i B_j, K^s_ij = int s B_i' B_j' with s(x) = sin(2 pi x) and the
// same (p+1)-point Gauss rule per element as M and K (bands as above).
void build_weighted_bands(Axis1D* A);

// Builds all of the above. reps: repeated interior breakpoints (k, e), 1 <= k
// <= n-1, 1 <= e <= p-1, each k at most once. Returns an empty string on
// success, else a message.
std::string build_axis(int n, int p, bool dir0, bool dir1, Axis1D* out,
                       const std::vector<std::pair<int, int>>& reps = {});

// Values and first derivatives of the kept B-splines of one direction at its
// n (p+1) Gauss points (the (p+1)-point rule of every element, element e
// owning points e (p+1) .. e (p+1) + p), for the general-coefficient
// stiffness: x, w (points and weights on [0, 1]); B and D as CSR matrices with
// one pattern (rows = points, at most p+1 columns each, increasing), and their
// transposes (rows = basis functions) with one pattern.
struct QuadAxis {
  int nq = 0, m = 0;
  std::vector<double> x, w;
  std::vector<int> rp, col;       // nq + 1 row pointers, column indices
  std::vector<double> bv, dv;     // B and D values on that pattern
  std::vector<int> trp, tcol;     // transpose: m + 1 row pointers, point indices
  std::vector<double> tbv, tdv;   // B^T and D^T values
};
void build_quad_axis(const Axis1D& A, QuadAxis* Q);

// Dense V_reg (m x n_reg, row-major) as the device passes apply it.
void expand_vreg(const Axis1D& A, double* V);

// Exact generalized eigendecomposition K q = lambda M q, Q^T M Q = I
// (dense, column-major Q: Q[i + j*m] = q_j[i]). Returns "" on success.
std::string exact_fd_axis(const Axis1D& ax, std::vector<double>* Q, std::vector<double>* lam);

// Symmetric cardinal B-spline B~_q at x = k/2 for integer k (exact recurrence).
double cardinal_half(int q, int twice_x);

// Radix decomposition of an FFT length: factors 8, 4, 2 first, then the odd
// prime factors in increasing order (3 and 5 have register butterflies, every
// other factor runs as a direct DFT stage).
bool fft_factor(int L, std::vector<int>* radices);

}  // namespace iffd
