/*
 * ORACLE (test infrastructure only).  Body of the reference schemes, compiled twice by
 * sigkernel_oracle.c: once with REAL = double (values) and once with REAL = double complex
 * (complex-step derivatives: d k / d x = Im k(x + i h e) / h, exact to rounding for these
 * rational maps).  Nothing here is blocked, fused or reordered: every scheme is written in the
 * physical coordinates (s, t) and in the order the paper states it.
 *
 * Expects the including file to define:
 *   REAL      the scalar type
 *   FN(name)  name mangling for this instantiation
 *   MAG(v)    a non-negative magnitude of v (used only for series stopping tests)
 */

/* r^n with the convention 0^0 = 1 (the paper's sums use (C dt)^0 = 1 for C = 0). */
static REAL FN(ipow)(REAL r, int n) {
    REAL v = 1.0;
    for (int i = 0; i < n; ++i) v *= r;
    return v;
}

/* <a, b> in R^d. */
static REAL FN(dot)(const REAL* a, const REAL* b, int d) {
    REAL v = 0.0;
    for (int c = 0; c < d; ++c) v += a[c] * b[c];
    return v;
}

/* Linear interpolation of a piecewise-linear path onto its lambda-order dyadic refinement:
 * every segment [u_i, u_{i+1}] is split into 2^lam equal pieces (Definition "dyadic scheme",
 * Section 2).  Output has lx*2^lam + 1 points. */
static REAL* FN(refine_path)(const REAL* x, int64_t L, int d, int lam) {
    int64_t R = (int64_t)1 << lam, lx = L - 1, n = lx * R + 1;
    REAL* xr = (REAL*)malloc(sizeof(REAL) * (size_t)(n * d));
    for (int64_t i = 0; i < lx; ++i)
        for (int64_t k = 0; k < R; ++k)
            for (int c = 0; c < d; ++c)
                xr[(i * R + k) * d + c] =
                    x[i * d + c] + ((double)k / (double)R) * (x[(i + 1) * d + c] - x[i * d + c]);
    for (int c = 0; c < d; ++c) xr[lx * R * d + c] = x[lx * d + c];
    return xr;
}

/* The matching refinement of a time partition (same construction on [s_i, s_{i+1}]). */
static double* FN(refine_grid)(const double* s, int64_t L, int lam) {
    int64_t R = (int64_t)1 << lam, lx = L - 1;
    double* sr = (double*)malloc(sizeof(double) * (size_t)(lx * R + 1));
    for (int64_t i = 0; i < lx; ++i)
        for (int64_t k = 0; k < R; ++k)
            sr[i * R + k] = s[i] + ((double)k / (double)R) * (s[i + 1] - s[i]);
    sr[lx * R] = s[lx];
    return sr;
}

/* ---------------------------------------------------------------------------------------------
 * Finite differences on the dyadic grid P_lambda (Definition "dyadic scheme", Section 2) with
 * the first-order explicit update (order 1), the second-order explicit update of eq.
 * (secondexplicitscheme), Remark "higherfd" (order 2), and the implicit update of Remark
 * "higherfd" (order 3).  The garbled arguments k(t_{i+1}, v_j) + k(t_i, v_{j+1}) in the
 * Definition are read as k(s_{i+1}, t_j) + k(s_i, t_{j+1}), the two nodes of the trapezoid rule
 * of Section 2.
 *
 * Implicit update.  The double integral of eq. (integralpde) over one sub-cell is taken by the
 * two-dimensional trapezoid rule on its four corners, (area/4) (k00 + k10 + k01 + k11), so with
 * m = C (s - u)(t - v):
 *     k11 = k10 + k01 - k00 + (m/4) (k00 + k10 + k01 + k11).
 * The Remark prints the factor as 1/2; with 1/2 a single cell from k = 1 on its edges gives
 * k11 = 1 + 2m + O(m^2) where the exact solution is 1 + m + m^2/4 + ..., so the factor is read
 * as the trapezoid rule's 1/4.  The equation is linear in k11 and is solved for it below; it
 * has no solution when m = 4 (the result is then inf or NaN).
 * ------------------------------------------------------------------------------------------- */
static REAL FN(fd)(const REAL* x, int64_t Lx, const REAL* y, int64_t Ly, int d, int order, int lam) {
    if (Lx < 2 || Ly < 2) return 1.0;
    REAL* xr = FN(refine_path)(x, Lx, d, lam);
    REAL* yr = FN(refine_path)(y, Ly, d, lam);
    int64_t nI = (Lx - 1) << lam, nJ = (Ly - 1) << lam;
    REAL* prev = (REAL*)malloc(sizeof(REAL) * (size_t)(nJ + 1)); /* k(s_u,   t_w) */
    REAL* cur = (REAL*)malloc(sizeof(REAL) * (size_t)(nJ + 1));  /* k(s_u+1, t_w) */
    REAL* dx = (REAL*)malloc(sizeof(REAL) * (size_t)d);
    REAL* dy = (REAL*)malloc(sizeof(REAL) * (size_t)d);
    for (int64_t w = 0; w <= nJ; ++w) prev[w] = 1.0; /* k(s_0, .) = 1 */
    for (int64_t u = 0; u < nI; ++u) {
        cur[0] = 1.0; /* k(., t_0) = 1 */
        for (int c = 0; c < d; ++c) dx[c] = xr[(u + 1) * d + c] - xr[u * d + c];
        for (int64_t w = 0; w < nJ; ++w) {
            for (int c = 0; c < d; ++c) dy[c] = yr[(w + 1) * d + c] - yr[w * d + c];
            REAL m = FN(dot)(dx, dy, d); /* <x_{s_u+1} - x_{s_u}, y_{t_w+1} - y_{t_w}> */
            REAL k10 = cur[w], k01 = prev[w + 1], k00 = prev[w];
            REAL v;
            if (order == 3) {
                v = (k10 + k01 - k00 + 0.25 * m * (k00 + k10 + k01)) / (1.0 - 0.25 * m);
            } else {
                v = k10 + k01 - k00 + 0.5 * m * (k10 + k01);
                if (order == 2) v += (1.0 / 12.0) * m * m * (k10 + k01 + k00);
            }
            cur[w + 1] = v;
        }
        REAL* tmp = prev; prev = cur; cur = tmp;
    }
    REAL out = prev[nJ];
    free(xr); free(yr); free(prev); free(cur); free(dx); free(dy);
    return out;
}

/* ---------------------------------------------------------------------------------------------
 * Polynomial approximation scheme of order N (Definition "def:polyapproxscheme", Section 3.2;
 * explicit update of the Remark that follows it).  p^{ij} and q^{ij} are the coefficients of the
 * bottom and left edges of cell (i,j) in powers of (s - s_i) and (t - t_j); the initial edges are
 * e_0 = (1, 0, ..., 0); the endpoint is the average of the two truncated edge evaluations.
 * Cells are visited row by row (i outer, j inner), a topological order of the recursion of
 * Definition "lambda".  The hybrid scheme of Section 3.2 (polynomial scheme on the dyadically
 * refined grid) is the same recursion applied to the refined paths and partitions.
 * ------------------------------------------------------------------------------------------- */
static REAL FN(poly_approx)(const REAL* x0, int64_t Lx0, const REAL* y0, int64_t Ly0, int d, int N,
                            int lam, const double* s0, const double* t0) {
    if (Lx0 < 2 || Ly0 < 2) return 1.0;
    double* su = s0 ? NULL : uniform_grid_(Lx0);
    double* tu = t0 ? NULL : uniform_grid_(Ly0);
    const double* sg = s0 ? s0 : su;
    const double* tg = t0 ? t0 : tu;
    REAL* x = FN(refine_path)(x0, Lx0, d, lam);
    REAL* y = FN(refine_path)(y0, Ly0, d, lam);
    double* s = FN(refine_grid)(sg, Lx0, lam);
    double* t = FN(refine_grid)(tg, Ly0, lam);
    int64_t lx = (Lx0 - 1) << lam, ly = (Ly0 - 1) << lam;

    double fact[80];
    fact[0] = 1.0;
    for (int k = 1; k < 80; ++k) fact[k] = fact[k - 1] * (double)k;

    REAL* q = (REAL*)calloc((size_t)(ly * (N + 1)), sizeof(REAL)); /* q^{i,j}, j = 0..ly-1 */
    REAL* p = (REAL*)malloc(sizeof(REAL) * (size_t)(N + 1));       /* p^{i,j} */
    REAL* pn = (REAL*)malloc(sizeof(REAL) * (size_t)(N + 1));
    REAL* qn = (REAL*)malloc(sizeof(REAL) * (size_t)(N + 1));
    REAL* dx = (REAL*)malloc(sizeof(REAL) * (size_t)d);
    REAL* dy = (REAL*)malloc(sizeof(REAL) * (size_t)d);
    for (int64_t j = 0; j < ly; ++j) q[j * (N + 1)] = 1.0; /* q^{0,j} = e_0 */

    for (int64_t i = 0; i < lx; ++i) {
        for (int n = 0; n <= N; ++n) p[n] = (n == 0) ? 1.0 : 0.0; /* p^{i,0} = e_0 */
        double ds = s[i + 1] - s[i];
        for (int c = 0; c < d; ++c) dx[c] = x[(i + 1) * d + c] - x[i * d + c];
        for (int64_t j = 0; j < ly; ++j) {
            double dt = t[j + 1] - t[j];
            for (int c = 0; c < d; ++c) dy[c] = y[(j + 1) * d + c] - y[j * d + c];
            REAL C = FN(dot)(dx, dy, d) / (ds * dt); /* C_ij */
            REAL* qj = q + j * (N + 1);
            for (int n = 0; n <= N; ++n) {
                REAL a = 0.0, b = 0.0;
                for (int k = 0; k <= n; ++k) {
                    a += p[k] * FN(ipow)(C * dt, n - k) * fact[k] / (fact[n - k] * fact[n]);
                    b += qj[k] * FN(ipow)(C * ds, n - k) * fact[k] / (fact[n - k] * fact[n]);
                }
                for (int k = 1; k <= N; ++k) {
                    a += qj[k] * FN(ipow)(C, n) * FN(ipow)(dt, n + k) * fact[k] / (fact[n + k] * fact[n]);
                    b += p[k] * FN(ipow)(C, n) * FN(ipow)(ds, n + k) * fact[k] / (fact[n + k] * fact[n]);
                }
                pn[n] = a; /* p^{i,j+1}_n */
                qn[n] = b; /* q^{i+1,j}_n */
            }
            for (int n = 0; n <= N; ++n) { p[n] = pn[n]; qj[n] = qn[n]; }
        }
    }
    /* p now holds p^{lx-1, ly}; q[ly-1] holds q^{lx, ly-1}. */
    double dsl = s[lx] - s[lx - 1], dtl = t[ly] - t[ly - 1];
    REAL end = 0.0;
    for (int n = 0; n <= N; ++n)
        end += p[n] * FN(ipow)(dsl, n) + q[(ly - 1) * (N + 1) + n] * FN(ipow)(dtl, n);
    end *= 0.5;
    free(q); free(p); free(pn); free(qn); free(dx); free(dy);
    free(x); free(y); free(s); free(t); free(su); free(tu);
    return end;
}

/* ---------------------------------------------------------------------------------------------
 * Polynomial interpolation scheme of order N (Definition "def:polyinterpscheme", Section 3.3).
 * Each cell keeps its closure: the interpolants g (bottom) and h (left) in powers of (s - s_i)
 * and (t - t_j), and C_ij.  Its solution is eq. (interpformula) of Proposition "propinterp":
 *   k(s,t) = g_0 0F1(1; z) + sum_{n=1..N} (g_n (s-s_i)^n + h_n (t-t_j)^n) 0F1(n+1; z),
 *   z = C_ij (s - s_i)(t - t_j),
 * with g_0 (the bottom interpolant's constant) in the first term exactly as printed.  The
 * incoming edges of cell (i,j) are the closures of cells (i,j-1) and (i-1,j) evaluated at the
 * N+1 Chebyshev extrema (eq. (chebextr) with m = 0..N, as Definition "interpooperator" asks for
 * N+1 points), interpolated by solving the Vandermonde system with partial-pivoting LU.
 * ------------------------------------------------------------------------------------------- */
typedef struct {
    REAL g[40], h[40];
    REAL C;
    double a, c; /* s_i, t_j */
} FN(closure);

/* 0F1(b; z) = sum_m z^m / ((b)_m m!) summed until the term is negligible (Prop. "propinterp"). */
static REAL FN(hyp0f1)(double b, REAL z) {
    REAL term = 1.0, sum = 1.0;
    for (int m = 0; m < 600; ++m) {
        term *= z / ((b + m) * (double)(m + 1));
        sum += term;
        if (MAG(term) <= 1e-19 * MAG(sum) || MAG(term) == 0.0) break;
    }
    return sum;
}

static REAL FN(closure_eval)(const FN(closure) * cl, int N, double s, double t) {
    double u = s - cl->a, v = t - cl->c;
    REAL z = cl->C * u * v;
    REAL k = cl->g[0] * FN(hyp0f1)(1.0, z);
    for (int n = 1; n <= N; ++n)
        k += (cl->g[n] * FN(ipow)(u, n) + cl->h[n] * FN(ipow)(v, n)) * FN(hyp0f1)((double)(n + 1), z);
    return k;
}

/* Solve V c = f for the (N+1)x(N+1) real matrix V (row-major), partial-pivoting LU. */
static void FN(solve_vandermonde)(const double* V0, const REAL* f, REAL* c, int n) {
    double V[41 * 41];
    REAL rhs[41];
    memcpy(V, V0, sizeof(double) * (size_t)(n * n));
    for (int r = 0; r < n; ++r) rhs[r] = f[r];
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(V[r * n + col]) > fabs(V[piv * n + col])) piv = r;
        if (piv != col) {
            for (int k = 0; k < n; ++k) {
                double tmp = V[col * n + k]; V[col * n + k] = V[piv * n + k]; V[piv * n + k] = tmp;
            }
            REAL tr = rhs[col]; rhs[col] = rhs[piv]; rhs[piv] = tr;
        }
        for (int r = col + 1; r < n; ++r) {
            double l = V[r * n + col] / V[col * n + col];
            for (int k = col; k < n; ++k) V[r * n + k] -= l * V[col * n + k];
            rhs[r] -= l * rhs[col];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        REAL acc = rhs[r];
        for (int k = r + 1; k < n; ++k) acc -= V[r * n + k] * c[k];
        c[r] = acc / V[r * n + r];
    }
}

static REAL FN(poly_interp)(const REAL* x0, int64_t Lx0, const REAL* y0, int64_t Ly0, int d, int N,
                            int lam, const double* s0, const double* t0) {
    if (Lx0 < 2 || Ly0 < 2) return 1.0;
    double* su = s0 ? NULL : uniform_grid_(Lx0);
    double* tu = t0 ? NULL : uniform_grid_(Ly0);
    const double* sg = s0 ? s0 : su;
    const double* tg = t0 ? t0 : tu;
    REAL* x = FN(refine_path)(x0, Lx0, d, lam);
    REAL* y = FN(refine_path)(y0, Ly0, d, lam);
    double* s = FN(refine_grid)(sg, Lx0, lam);
    double* t = FN(refine_grid)(tg, Ly0, lam);
    int64_t lx = (Lx0 - 1) << lam, ly = (Ly0 - 1) << lam;
    const double PI = 3.14159265358979323846;

    FN(closure)* below = (FN(closure)*)calloc((size_t)ly, sizeof(FN(closure))); /* row i-1 */
    FN(closure)* row = (FN(closure)*)calloc((size_t)ly, sizeof(FN(closure)));   /* row i   */
    REAL* dx = (REAL*)malloc(sizeof(REAL) * (size_t)d);
    REAL* dy = (REAL*)malloc(sizeof(REAL) * (size_t)d);
    double V[41 * 41], nodes[41];
    REAL vals[41];

    for (int64_t i = 0; i < lx; ++i) {
        double ds = s[i + 1] - s[i];
        for (int c = 0; c < d; ++c) dx[c] = x[(i + 1) * d + c] - x[i * d + c];
        for (int64_t j = 0; j < ly; ++j) {
            double dt = t[j + 1] - t[j];
            for (int c = 0; c < d; ++c) dy[c] = y[(j + 1) * d + c] - y[j * d + c];
            FN(closure)* cl = &row[j];
            cl->a = s[i];
            cl->c = t[j];
            cl->C = FN(dot)(dx, dy, d) / (ds * dt);
            /* Omega^N of the bottom edge sigma_ij = k(., t_j) on [s_i, s_{i+1}]. */
            for (int m = 0; m <= N; ++m) {
                nodes[m] = 0.5 * ds * cos(PI * m / N) + 0.5 * (s[i] + s[i + 1]);
                vals[m] = (j == 0) ? (REAL)1.0 : FN(closure_eval)(&row[j - 1], N, nodes[m], t[j]);
                for (int n = 0; n <= N; ++n) V[m * (N + 1) + n] = pow(nodes[m] - s[i], n);
            }
            FN(solve_vandermonde)(V, vals, cl->g, N + 1);
            /* Omega^N of the left edge tau_ij = k(s_i, .) on [t_j, t_{j+1}]. */
            for (int m = 0; m <= N; ++m) {
                nodes[m] = 0.5 * dt * cos(PI * m / N) + 0.5 * (t[j] + t[j + 1]);
                vals[m] = (i == 0) ? (REAL)1.0 : FN(closure_eval)(&below[j], N, s[i], nodes[m]);
                for (int n = 0; n <= N; ++n) V[m * (N + 1) + n] = pow(nodes[m] - t[j], n);
            }
            FN(solve_vandermonde)(V, vals, cl->h, N + 1);
        }
        FN(closure)* tmp = below; below = row; row = tmp;
    }
    /* Endpoint: average of sigma_{lx-1,ly}(s_lx) and tau_{lx,ly-1}(t_ly); both are the closure of
     * the last cell evaluated at its top-right corner. */
    const FN(closure)* last = &below[ly - 1];
    REAL top = FN(closure_eval)(last, N, s[lx], t[ly]);
    REAL right = FN(closure_eval)(last, N, s[lx], t[ly]);
    REAL end = 0.5 * (top + right);
    free(below); free(row); free(dx); free(dy);
    free(x); free(y); free(s); free(t); free(su); free(tu);
    return end;
}

/* Dispatch on the scheme id: 0 FD1, 1 FD2, 2 polynomial approximation, 3 interpolation,
 * 4 implicit FD. */
static REAL FN(scheme)(int scheme, const REAL* x, int64_t Lx, const REAL* y, int64_t Ly, int d,
                       int N, int lam, const double* s, const double* t) {
    switch (scheme) {
        case 0: return FN(fd)(x, Lx, y, Ly, d, 1, lam);
        case 1: return FN(fd)(x, Lx, y, Ly, d, 2, lam);
        case 2: return FN(poly_approx)(x, Lx, y, Ly, d, N, lam, s, t);
        case 3: return FN(poly_interp)(x, Lx, y, Ly, d, N, lam, s, t);
        case 4: return FN(fd)(x, Lx, y, Ly, d, 3, lam);
        default: return 0.0 / 0.0;
    }
}
