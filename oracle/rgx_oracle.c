/*
 * rgx_oracle.c -- plain FP64 CPU reference for differentiable volume ray
 * marching through truncated elliptical Gaussians (RayGaussX, arXiv 2509.07782).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or execute this file; only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark do.  It shares no code, header, table or
 * constant with the CUDA implementation.
 *
 * What it computes, and where the paper defines it:
 *   - density / radiance fields ............ Eq. 1 (Sec. 3.1)
 *   - truncated Gaussian, sigma_eps ellipsoid  Supp. Sec. 2.1 (Eq. of sigma_l, Sigma = R S S^T R^T)
 *   - ray-marching discretisation .......... Eq. 3 (Sec. 3.1)
 *   - segment loop, ClosestHit skipping .... Algorithm 1, Eq. 4 (Sec. 3.2)
 *   - adaptive segment size ................ Eq. 5 (Sec. 3.2)
 *   - minimal AABB half-lengths ............ Supp. Sec. 2.2 (Cauchy-Schwarz result)
 *   - real spherical harmonics ............. Eq. 1's c_l(d) (SH appearance, Supp. Sec. 6.1)
 *   - spherical-Gaussian lobes ............. Eq. 1's c_l(d) "with SH/SG" (Sec. 3.1); Supp.
 *                                            Sec. 6.1 uses nine SH and seven SG per primitive
 *   - adjoint of Eq. 3 ..................... derived here; the paper trains through
 *                                            the renderer (Sec. 3.5) but prints no
 *                                            derivation.
 *
 * Readings where the paper is silent, ambiguous or leaves a choice open:
 *   - hard truncation per sample: a Gaussian contributes only where
 *     q(x) <= Q_eps = 2 ln(sigma~/sigma_eps);
 *   - samples sit at segment midpoints t_S + (k + 1/2) dt;
 *   - uniform mode + skipping snaps the segment start to the lattice
 *     t_n + j dt (one step of guard) so that skipping moves no sample;
 *   - the hit set of a segment [t_S, t_S+dS) is every Gaussian whose ellipsoid
 *     chord [t_in, t_out] overlaps it (segments lying wholly inside an ellipsoid
 *     count, Supp. Sec. 6.2);
 *   - colour activation c_l(d) = max(0, 1/2 + sum_k Y_k(d) K_lk
 *     + sum_j a_lj exp(lambda_lj (mu_lj . d - 1))), d the ray direction; lobe j
 *     has a raw axis normalised here (mu = u / |u|), a sharpness lambda >= 0 and
 *     an RGB amplitude a, stored as 7 numbers (u_x, u_y, u_z, lambda, a_r, a_g, a_b);
 *   - truncation boundary, schedule and termination are piecewise constant in
 *     the adjoint (stop-gradient).
 *
 * Everything is brute force: every ray solves the chord of every Gaussian.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OX_OK 0
#define OX_ERR_ARG 1
#define OX_ERR_ITER 2
#define OX_ERR_MEM 3

typedef struct {
    double c2w[12];            /* row-major 3x4, column 3 = camera centre */
    double fx, fy, cx, cy;
    int32_t width, height;
    double t_near, t_far;      /* t_far <= 0: exit of the scene bounding box */
} ox_camera;

typedef struct {
    int32_t skip;              /* Alg. 1 ClosestHit skipping */
    int32_t adaptive;          /* Eq. 5 */
    int32_t n_s;               /* samples per segment */
    int32_t max_segments;      /* loop bound (0: none) */
    double dt;                 /* uniform step */
    double dt_min, dt_max, beta;
    double t_eps;              /* transmittance threshold T_eps */
    double sigma_eps;          /* truncation density */
    double bg[3];
} ox_opts;

/* ------------------------------------------------------------------------ */
/* per-Gaussian set-up                                                       */
/* ------------------------------------------------------------------------ */

/* Rotation matrix of the unit quaternion (w, x, y, z) (textbook formula). */
void ox_quat_to_rot(const double q[4], double R[9])
{
    double n = sqrt(q[0]*q[0] + q[1]*q[1] + q[2]*q[2] + q[3]*q[3]);
    double w = q[0]/n, x = q[1]/n, y = q[2]/n, z = q[3]/n;
    R[0] = 1 - 2*(y*y + z*z); R[1] = 2*(x*y - w*z);     R[2] = 2*(x*z + w*y);
    R[3] = 2*(x*y + w*z);     R[4] = 1 - 2*(x*x + z*z); R[5] = 2*(y*z - w*x);
    R[6] = 2*(x*z - w*y);     R[7] = 2*(y*z + w*x);     R[8] = 1 - 2*(x*x + y*y);
}

typedef struct {
    double mu[3];
    double M[9];      /* S^-1 R^T : y = M (x - mu), q = |y|^2 = (x-mu)^T Sigma^-1 (x-mu) */
    double R[9];
    double s[3];
    double sig;       /* sigma~ */
    double Qe;        /* 2 ln(sigma~ / sigma_eps); <= 0 means empty support */
    double K[16][3];
    int nk;
    const double* sg; /* nsg lobes x (u_x, u_y, u_z, lambda, a_r, a_g, a_b), or NULL */
    int nsg;
} ox_prim;

static void prim_setup(ox_prim* p, const double* mu, const double* s, const double* q,
                       double sig, const double* sh, int nk, double sigma_eps)
{
    for (int i = 0; i < 3; i++) { p->mu[i] = mu[i]; p->s[i] = s[i]; }
    ox_quat_to_rot(q, p->R);
    for (int j = 0; j < 3; j++)
        for (int k = 0; k < 3; k++)
            p->M[3*j + k] = p->R[3*k + j] / s[j];
    p->sig = sig;
    p->Qe = (sig > sigma_eps) ? 2.0 * log(sig / sigma_eps) : 0.0;
    p->nk = nk;
    for (int k = 0; k < 16; k++)
        for (int c = 0; c < 3; c++)
            p->K[k][c] = (k < nk) ? sh[3*k + c] : 0.0;
    p->sg = NULL;
    p->nsg = 0;
}

/* Half-lengths of the minimal AABB of the sigma_eps ellipsoid:
 * L_i = sqrt(sum_j r_ij^2 s~_j^2), s~_j = sqrt(Q_eps) s_j (Supp. Sec. 2.2). */
void ox_prim_geometry(int64_t n, const double* means, const double* scales, const double* quats,
                      const double* dens, double sigma_eps,
                      double* R_out, double* M_out, double* Qe_out, double* half_out)
{
    for (int64_t l = 0; l < n; l++) {
        ox_prim p;
        prim_setup(&p, means + 3*l, scales + 3*l, quats + 4*l, dens[l], NULL, 0, sigma_eps);
        if (R_out) memcpy(R_out + 9*l, p.R, sizeof p.R);
        if (M_out) memcpy(M_out + 9*l, p.M, sizeof p.M);
        if (Qe_out) Qe_out[l] = p.Qe;
        if (half_out) {
            for (int i = 0; i < 3; i++) {
                double acc = 0;
                for (int j = 0; j < 3; j++) {
                    double st = sqrt(p.Qe) * p.s[j];
                    acc += p.R[3*i + j] * p.R[3*i + j] * st * st;
                }
                half_out[3*l + i] = sqrt(acc);
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* real spherical harmonics from the normalisation formula                   */
/* ------------------------------------------------------------------------ */

static double factorial(int k) { double f = 1; for (int i = 2; i <= k; i++) f *= i; return f; }

/* Associated Legendre P_l^m(x), m >= 0, with the Condon-Shortley phase. */
static double assoc_legendre(int l, int m, double x)
{
    double pmm = 1.0;
    if (m > 0) {
        double sx = sqrt((1.0 - x) * (1.0 + x)), f = 1.0;
        for (int i = 1; i <= m; i++) { pmm *= -f * sx; f += 2.0; }
    }
    if (l == m) return pmm;
    double pm1 = x * (2*m + 1) * pmm;
    if (l == m + 1) return pm1;
    double pll = 0;
    for (int ll = m + 2; ll <= l; ll++) {
        pll = ((2*ll - 1) * x * pm1 - (ll + m - 1) * pmm) / (ll - m);
        pmm = pm1; pm1 = pll;
    }
    return pll;
}

/* Real SH Y_k(d), k = l^2 + l + m, l <= deg:
 *   m > 0: sqrt2 K_l^m cos(m phi) P_l^m(cos th)
 *   m < 0: sqrt2 K_l^|m| sin(|m| phi) P_l^|m|(cos th)
 *   m = 0: K_l^0 P_l^0(cos th)
 * with K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!). */
void ox_sh_basis(int deg, const double d[3], double* Y)
{
    double nrm = sqrt(d[0]*d[0] + d[1]*d[1] + d[2]*d[2]);
    double x = d[0]/nrm, y = d[1]/nrm, z = d[2]/nrm;
    double phi = atan2(y, x);
    for (int l = 0; l <= deg; l++) {
        for (int m = -l; m <= l; m++) {
            int am = m < 0 ? -m : m;
            double K = sqrt((2.0*l + 1.0) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
            double P = assoc_legendre(l, am, z);
            double v;
            if (m > 0) v = sqrt(2.0) * K * cos(am * phi) * P;
            else if (m < 0) v = sqrt(2.0) * K * sin(am * phi) * P;
            else v = K * P;
            Y[l*l + l + m] = v;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* rays, chords, closest hit                                                 */
/* ------------------------------------------------------------------------ */

static void make_ray(const ox_camera* cam, int64_t pix, double o[3], double d[3])
{
    int64_t u = pix % cam->width, v = pix / cam->width;
    double dc[3] = { ((double)u + 0.5 - cam->cx) / cam->fx, ((double)v + 0.5 - cam->cy) / cam->fy, 1.0 };
    for (int r = 0; r < 3; r++) {
        o[r] = cam->c2w[4*r + 3];
        d[r] = cam->c2w[4*r + 0]*dc[0] + cam->c2w[4*r + 1]*dc[1] + cam->c2w[4*r + 2]*dc[2];
    }
    double n = sqrt(d[0]*d[0] + d[1]*d[1] + d[2]*d[2]);
    for (int r = 0; r < 3; r++) d[r] /= n;
}

/* Chord of the ray with the Q_eps ellipsoid: roots of |M(o + t d - mu)|^2 = Q_eps.
 * Returns 1 and [t_in, t_out] when the chord has positive length. */
static int chord(const ox_prim* p, const double o[3], const double d[3], double* tin, double* tout)
{
    if (p->Qe <= 0) return 0;
    double y0[3], yd[3];
    for (int j = 0; j < 3; j++) {
        y0[j] = p->M[3*j]*(o[0]-p->mu[0]) + p->M[3*j+1]*(o[1]-p->mu[1]) + p->M[3*j+2]*(o[2]-p->mu[2]);
        yd[j] = p->M[3*j]*d[0] + p->M[3*j+1]*d[1] + p->M[3*j+2]*d[2];
    }
    double a = yd[0]*yd[0] + yd[1]*yd[1] + yd[2]*yd[2];
    double b = y0[0]*yd[0] + y0[1]*yd[1] + y0[2]*yd[2];
    double c = y0[0]*y0[0] + y0[1]*y0[1] + y0[2]*y0[2] - p->Qe;
    double disc = b*b - a*c;
    if (!(disc > 0) || !(a > 0)) return 0;
    double sq = sqrt(disc);
    *tin = (-b - sq) / a;
    *tout = (-b + sq) / a;
    return 1;
}

typedef struct { int64_t l; double tin, tout; } ox_chord;

/* ClosestHit(t_a): min over chords with t_out > t_a and t_in < t_f of max(t_in, t_a);
 * t_f when there is none (Alg. 1, Eq. 4). */
static double closest_hit(const ox_chord* ch, int64_t nch, double ta, double tf)
{
    double best = tf;
    for (int64_t i = 0; i < nch; i++) {
        if (ch[i].tout > ta && ch[i].tin < tf) {
            double t = ch[i].tin > ta ? ch[i].tin : ta;
            if (t < best) best = t;
        }
    }
    return best;
}

/* Scene bounding box: union of the per-Gaussian minimal AABBs. */
static void scene_box(const ox_prim* P, int64_t n, double lo[3], double hi[3])
{
    for (int i = 0; i < 3; i++) { lo[i] = INFINITY; hi[i] = -INFINITY; }
    for (int64_t l = 0; l < n; l++) {
        if (P[l].Qe <= 0) continue;
        for (int i = 0; i < 3; i++) {
            double acc = 0;
            for (int j = 0; j < 3; j++) {
                double st = sqrt(P[l].Qe) * P[l].s[j];
                acc += P[l].R[3*i+j] * P[l].R[3*i+j] * st * st;
            }
            double L = sqrt(acc);
            if (P[l].mu[i] - L < lo[i]) lo[i] = P[l].mu[i] - L;
            if (P[l].mu[i] + L > hi[i]) hi[i] = P[l].mu[i] + L;
        }
    }
}

/* Far bound of a ray: camera t_far, or the exit of the scene box. */
static double far_bound(const ox_camera* cam, const double lo[3], const double hi[3],
                        const double o[3], const double d[3], double tn)
{
    if (cam->t_far > 0) return cam->t_far;
    if (!(lo[0] <= hi[0] && lo[1] <= hi[1] && lo[2] <= hi[2])) return tn;   /* empty scene */
    double t0 = -INFINITY, t1 = INFINITY;
    for (int i = 0; i < 3; i++) {
        if (d[i] != 0) {
            double a = (lo[i] - o[i]) / d[i], b = (hi[i] - o[i]) / d[i];
            if (a > b) { double t = a; a = b; b = t; }
            if (a > t0) t0 = a;
            if (b < t1) t1 = b;
        } else if (o[i] < lo[i] || o[i] > hi[i]) {
            return tn;
        }
    }
    if (t1 < t0 || t1 < tn) return tn;
    return t1;
}

/* ------------------------------------------------------------------------ */
/* the march (Alg. 1)                                                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    /* outputs */
    double C[3], T;
    int64_t nseg;          /* evaluated segments */
    int64_t active;        /* (sample, Gaussian) pairs inside the truncation */
    uint64_t active_hash;  /* order-free checksum of that set */
    int err;
} ox_ray_out;

/* One recorded evaluated segment: start, per-sample step, number of samples. */
typedef struct { double tS, dtk; } ox_seg;

/* Sample record used by the adjoint. */
typedef struct { double dtk, T, sigma, c[3]; int64_t first, count; } ox_sample;
typedef struct { int64_t l; double g; double t; } ox_contrib;

typedef struct {
    ox_sample* S; int64_t nS, capS;
    ox_contrib* G; int64_t nG, capG;
} ox_tape;

static void tape_push_sample(ox_tape* tp, ox_sample s)
{
    if (tp->nS == tp->capS) { tp->capS = tp->capS ? 2*tp->capS : 256; tp->S = realloc(tp->S, tp->capS * sizeof *tp->S); }
    tp->S[tp->nS++] = s;
}
static void tape_push_contrib(ox_tape* tp, ox_contrib c)
{
    if (tp->nG == tp->capG) { tp->capG = tp->capG ? 2*tp->capG : 1024; tp->G = realloc(tp->G, tp->capG * sizeof *tp->G); }
    tp->G[tp->nG++] = c;
}

/* Evaluate the samples of one segment, Eq. 1 + Eq. 3.  `hits` is the hit set
 * (indices into ch).  If brute != 0 every Gaussian of the scene is evaluated at
 * every sample instead.  Colours cl[l] were computed per (ray, Gaussian). */
static void prim_colour(const ox_prim* p, const double Y[16], const double d[3], double c[3], double pre[3]);

static void eval_segment(const ox_prim* P, int64_t nP, const ox_chord* ch, const int64_t* hits,
                         int64_t nh, const double (*colour)[3], const int64_t* ch_of_prim,
                         const double Ybasis[16],
                         const double o[3], const double d[3], double tS, double dtk, int ns, double tf,
                         int brute, ox_ray_out* out, ox_tape* tape)
{
    for (int k = 0; k < ns; k++) {
        double t = tS + (k + 0.5) * dtk;
        if (!(t < tf)) break;
        double x[3] = { o[0] + t*d[0], o[1] + t*d[1], o[2] + t*d[2] };
        double sigma = 0, S[3] = {0, 0, 0};
        int64_t first = tape ? tape->nG : 0, count = 0;
        int64_t nloop = brute ? nP : nh;
        for (int64_t h = 0; h < nloop; h++) {
            int64_t l = brute ? h : ch[hits[h]].l;
            const ox_prim* p = &P[l];
            if (p->Qe <= 0) continue;
            double y[3], q = 0;
            for (int j = 0; j < 3; j++) {
                y[j] = p->M[3*j]*(x[0]-p->mu[0]) + p->M[3*j+1]*(x[1]-p->mu[1]) + p->M[3*j+2]*(x[2]-p->mu[2]);
                q += y[j]*y[j];
            }
            if (!(q <= p->Qe)) continue;      /* hard truncation */
            double g = p->sig * exp(-0.5 * q);
            double ctmp[3];
            const double* c;
            if (brute) {
                /* a Gaussian without a chord can only be touched at tangency */
                if (ch_of_prim[l] >= 0) c = colour[ch_of_prim[l]];
                else { double pre[3]; prim_colour(p, Ybasis, d, ctmp, pre); c = ctmp; }
            } else {
                c = colour[hits[h]];
            }
            sigma += g;
            for (int r = 0; r < 3; r++) S[r] += g * c[r];
            out->active++;
            out->active_hash += (uint64_t)(l + 1) * 1000003ULL + (uint64_t)k * 7919ULL
                              + (uint64_t)llround(tS * 1e6);
            if (tape) { ox_contrib cc = { l, g, t }; tape_push_contrib(tape, cc); count++; }
        }
        if (sigma > 0) {
            double e = exp(-sigma * dtk);
            double alpha = 1.0 - e;
            double ci[3] = { S[0]/sigma, S[1]/sigma, S[2]/sigma };
            if (tape) {
                ox_sample s = { dtk, out->T, sigma, { ci[0], ci[1], ci[2] }, first, count };
                tape_push_sample(tape, s);
            }
            for (int r = 0; r < 3; r++) out->C[r] += out->T * alpha * ci[r];
            out->T *= e;
        }
    }
}

/* Value exp(lambda (mu . d - 1)) of spherical-Gaussian lobe j of p along d, with
 * mu = u / |u| its unit axis; also returns mu . d. */
static double sg_lobe(const ox_prim* p, int j, const double d[3], double* cosv)
{
    const double* r = p->sg + 7*j;
    double nu = sqrt(r[0]*r[0] + r[1]*r[1] + r[2]*r[2]);
    double cd = (r[0]*d[0] + r[1]*d[1] + r[2]*d[2]) / nu;
    if (cosv) *cosv = cd;
    return exp(r[3] * (cd - 1.0));
}

/* Colour of Gaussian p seen along direction d:
 * max(0, 1/2 + sum_k Y_k(d) K_k + sum_j a_j exp(lambda_j (mu_j . d - 1))). */
static void prim_colour(const ox_prim* p, const double Y[16], const double d[3], double c[3], double pre[3])
{
    for (int r = 0; r < 3; r++) {
        double acc = 0.5;
        for (int k = 0; k < p->nk; k++) acc += Y[k] * p->K[k][r];
        pre[r] = acc;
    }
    for (int j = 0; j < p->nsg; j++) {
        double e = sg_lobe(p, j, d, NULL);
        for (int r = 0; r < 3; r++) pre[r] += p->sg[7*j + 4 + r] * e;
    }
    for (int r = 0; r < 3; r++) c[r] = pre[r] > 0 ? pre[r] : 0;
}

/* March one ray.  sched_in (replay) gives the evaluated segments to use
 * instead of taking decisions; sched_out records them. */
static void march_ray(const ox_prim* P, int64_t nP, int sh_deg, const ox_camera* cam, const ox_opts* op,
                      const double lo[3], const double hi[3], int64_t pix,
                      int brute, const ox_seg* sched_in, int64_t nsched_in,
                      ox_seg* sched_out, int64_t sched_cap, int64_t* nsched_out,
                      ox_ray_out* out, ox_tape* tape,
                      double* o_out, double* d_out)
{
    double o[3], d[3];
    make_ray(cam, pix, o, d);
    if (o_out) memcpy(o_out, o, sizeof o);
    if (d_out) memcpy(d_out, d, sizeof d);
    memset(out, 0, sizeof *out);
    out->T = 1.0;

    double tn = cam->t_near;
    double tf = far_bound(cam, lo, hi, o, d, tn);

    /* brute-force chords of every Gaussian */
    ox_chord* ch = malloc((size_t)(nP > 0 ? nP : 1) * sizeof *ch);
    int64_t nch = 0;
    int64_t* ch_of_prim = brute ? malloc((size_t)(nP > 0 ? nP : 1) * sizeof(int64_t)) : NULL;
    for (int64_t l = 0; l < nP; l++) {
        double a, b;
        if (ch_of_prim) ch_of_prim[l] = -1;
        if (chord(&P[l], o, d, &a, &b)) {
            if (ch_of_prim) ch_of_prim[l] = nch;
            ch[nch].l = l; ch[nch].tin = a; ch[nch].tout = b; nch++;
        }
    }
    double Y[16];
    ox_sh_basis(sh_deg, d, Y);
    double (*colour)[3] = malloc((size_t)(nch > 0 ? nch : 1) * sizeof *colour);
    for (int64_t i = 0; i < nch; i++) {
        double pre[3];
        prim_colour(&P[ch[i].l], Y, d, colour[i], pre);
    }
    int64_t* hits = malloc((size_t)(nch > 0 ? nch : 1) * sizeof(int64_t));
    int64_t nrec = 0;

    if (sched_in) {
        /* replay: evaluate exactly the given segments, hit set = all chords */
        for (int64_t i = 0; i < nch; i++) hits[i] = i;
        for (int64_t s = 0; s < nsched_in; s++) {
            eval_segment(P, nP, ch, hits, nch, (const double (*)[3])colour, ch_of_prim, Y, o, d,
                         sched_in[s].tS, sched_in[s].dtk, op->n_s, tf, brute, out, tape);
            out->nseg++;
        }
    } else {
        const int ns = op->n_s;
        const int uniform = !op->adaptive;
        double tS = tn;
        int64_t j = 0;                         /* lattice index in uniform mode */
        if (op->skip) {
            double th = closest_hit(ch, nch, tn, tf);
            if (uniform) {
                int64_t jj = (int64_t)floor((th - tn) / op->dt) - 1;
                j = jj > 0 ? jj : 0;
                tS = tn + j * op->dt;
            } else {
                tS = th;
            }
        }
        int64_t iters = 0;
        while (tS < tf && out->T > op->t_eps) {
            if (op->max_segments > 0 && iters >= op->max_segments) { out->err = OX_ERR_ITER; break; }
            iters++;
            double dS, dtk;
            if (uniform) {
                dtk = op->dt;
                dS = ns * op->dt;
            } else {
                double a = tS / op->beta;
                if (a < op->dt_min) a = op->dt_min;
                a *= pow(out->T, -1.0 / 3.0);
                if (a > op->dt_max) a = op->dt_max;
                dtk = a;
                dS = ns * a;
            }
            double te = uniform ? tn + (j + ns) * op->dt : tS + dS;
            double tcut = te < tf ? te : tf;
            int64_t nh = 0;
            for (int64_t i = 0; i < nch; i++)
                if (ch[i].tin < tcut && ch[i].tout > tS) hits[nh++] = i;
            if (nh == 0) {
                if (op->skip) {
                    double th = closest_hit(ch, nch, te, tf);
                    if (uniform) {
                        int64_t jj = (int64_t)floor((th - tn) / op->dt) - 1;
                        j = jj > j + 1 ? jj : j + 1;
                        tS = tn + j * op->dt;
                    } else {
                        tS = th;
                    }
                } else {
                    if (uniform) { j += ns; tS = tn + j * op->dt; } else tS = te;
                }
                continue;
            }
            if (sched_out && nrec < sched_cap) { sched_out[nrec].tS = tS; sched_out[nrec].dtk = dtk; }
            nrec++;
            eval_segment(P, nP, ch, hits, nh, (const double (*)[3])colour, ch_of_prim, Y, o, d,
                         tS, dtk, ns, tf, brute, out, tape);
            out->nseg++;
            if (uniform) { j += ns; tS = tn + j * op->dt; } else tS = te;
        }
    }
    if (nsched_out) *nsched_out = nrec;
    free(ch); free(colour); free(hits); free(ch_of_prim);
}

static ox_prim* setup_all(int64_t n, const double* means, const double* scales, const double* quats,
                          const double* dens, const double* sh, int sh_deg, int nsg, const double* sg,
                          double sigma_eps)
{
    int nk = (sh_deg + 1) * (sh_deg + 1);
    ox_prim* P = malloc((size_t)(n > 0 ? n : 1) * sizeof *P);
    if (!P) return NULL;
    #pragma omp parallel for schedule(static)
    for (int64_t l = 0; l < n; l++) {
        prim_setup(&P[l], means + 3*l, scales + 3*l, quats + 4*l, dens[l], sh + (int64_t)nk*3*l, nk, sigma_eps);
        if (nsg > 0 && sg) { P[l].sg = sg + (int64_t)7*nsg*l; P[l].nsg = nsg; }
    }
    return P;
}

static int set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads; return 1;
#endif
}

/*
 * Forward render.  pix == NULL renders every pixel of the camera (npix must be
 * width*height).  rgba[npix*4] = (C + T bg, 1 - T); state[npix*4] = (C, T);
 * nseg[npix]; active[npix*2] = (count, checksum) of in-support (sample,
 * Gaussian) pairs.  sched_* record (or, with replay != 0, supply) the evaluated
 * segments (tS, dt_k) of every ray, sched_cap per ray.
 * Returns the number of rays that hit the segment limit (0 when none).
 */
int64_t ox_render(int64_t n, const double* means, const double* scales, const double* quats,
                  const double* dens, const double* sh, int32_t sh_deg, int32_t n_sg, const double* sg,
                  const ox_camera* cam, const ox_opts* op,
                  int64_t npix, const int64_t* pix,
                  double* rgba, double* state, int64_t* nseg, int64_t* active,
                  int64_t sched_cap, double* sched, int64_t* sched_n, int32_t replay,
                  int32_t brute, int32_t nthreads)
{
    set_threads(nthreads);
    if (n_sg < 0 || n_sg > 7 || (n_sg > 0 && !sg)) return -1;
    ox_prim* P = setup_all(n, means, scales, quats, dens, sh, sh_deg, n_sg, sg, op->sigma_eps);
    if (!P) return -1;
    double lo[3], hi[3];
    scene_box(P, n, lo, hi);
    int64_t nerr = 0;
    #pragma omp parallel for schedule(dynamic, 4) reduction(+:nerr)
    for (int64_t i = 0; i < npix; i++) {
        int64_t p = pix ? pix[i] : i;
        ox_ray_out r;
        ox_seg* sin_ = NULL; int64_t nsin = 0;
        ox_seg* sout = NULL;
        if (sched && replay) { sin_ = (ox_seg*)(sched + 2*sched_cap*i); nsin = sched_n[i]; }
        if (sched && !replay) sout = (ox_seg*)(sched + 2*sched_cap*i);
        int64_t nrec = 0;
        march_ray(P, n, sh_deg, cam, op, lo, hi, p, brute, sin_, nsin, sout, sched_cap, &nrec, &r, NULL, NULL, NULL);
        if (sched && !replay) sched_n[i] = nrec;
        rgba[4*i + 0] = r.C[0] + r.T * op->bg[0];
        rgba[4*i + 1] = r.C[1] + r.T * op->bg[1];
        rgba[4*i + 2] = r.C[2] + r.T * op->bg[2];
        rgba[4*i + 3] = 1.0 - r.T;
        if (state) { state[4*i] = r.C[0]; state[4*i+1] = r.C[1]; state[4*i+2] = r.C[2]; state[4*i+3] = r.T; }
        if (nseg) nseg[i] = r.nseg;
        if (active) { active[2*i] = r.active; active[2*i+1] = (int64_t)r.active_hash; }
        if (r.err) nerr++;
    }
    free(P);
    return nerr;
}

/* ------------------------------------------------------------------------ */
/* adjoint                                                                   */
/* ------------------------------------------------------------------------ */

static void atomic_add(double* a, double v)
{
    #pragma omp atomic
    *a += v;
}

/*
 * Analytic gradient of L = sum_p <d_rgba[p], rgba[p]> with respect to means,
 * scales, quats (raw, unnormalised), densities and SH coefficients, on the
 * natural schedule of each ray (discrete decisions held fixed).  Gradients
 * are ADDED into the output arrays (caller zeroes them).
 *
 * For the samples i of a ray (Eq. 3) with T_{i+1} = T_i e^{-sigma_i dt_i},
 * alpha_i = 1 - e^{-sigma_i dt_i}, c_i = S_i / sigma_i, outputs
 * RGB = C + T_f bg, A = 1 - T_f, upstream a = dL/dRGB, b = dL/dA:
 *   dL/dT_f     = a.bg - b
 *   dL/dsigma_i = dt_i [ a.(T_{i+1} c_i - (C - C_{<=i})) - (a.bg - b) T_f ]
 *   dL/dc_i     = a T_i alpha_i
 * and for each Gaussian l active at sample i with g_l = sigma~_l exp(-q_l/2):
 *   dL/dg_l    = dL/dsigma_i + dL/dc_i . (c_l - c_i) / sigma_i
 *   dL/dc_l   += dL/dc_i g_l / sigma_i
 *   dg/dsigma~ = g / sigma~,  dg/dmu = g Sigma^-1 (x - mu),  dg/dM = -g y (x-mu)^T
 * with M = S^-1 R^T, chained to s, R(q^) and q.
 */
int64_t ox_backward(int64_t n, const double* means, const double* scales, const double* quats,
                    const double* dens, const double* sh, int32_t sh_deg, int32_t n_sg, const double* sg,
                    const ox_camera* cam, const ox_opts* op,
                    int64_t npix, const int64_t* pix, const double* d_rgba,
                    double* g_means, double* g_scales, double* g_quats, double* g_dens, double* g_sh,
                    double* g_sg, int32_t nthreads)
{
    set_threads(nthreads);
    int nk = (sh_deg + 1) * (sh_deg + 1);
    if (n_sg < 0 || n_sg > 7 || (n_sg > 0 && (!sg || !g_sg))) return -1;
    ox_prim* P = setup_all(n, means, scales, quats, dens, sh, sh_deg, n_sg, sg, op->sigma_eps);
    if (!P) return -1;
    double lo[3], hi[3];
    scene_box(P, n, lo, hi);
    /* dL/dM and dL/dmu etc. are accumulated per Gaussian, then chained to s, q */
    double* gM = calloc((size_t)(n > 0 ? n : 1) * 9, sizeof(double));
    int64_t nerr = 0;

    #pragma omp parallel for schedule(dynamic, 4) reduction(+:nerr)
    for (int64_t i = 0; i < npix; i++) {
        const double* up = d_rgba + 4*i;
        if (up[0] == 0 && up[1] == 0 && up[2] == 0 && up[3] == 0) continue;
        int64_t p = pix ? pix[i] : i;
        ox_ray_out r;
        ox_tape tape = {0};
        double o[3], d[3];
        march_ray(P, n, sh_deg, cam, op, lo, hi, p, 0, NULL, 0, NULL, 0, NULL, &r, &tape, o, d);
        if (r.err) nerr++;
        double a[3] = { up[0], up[1], up[2] }, b = up[3];
        double dTf = a[0]*op->bg[0] + a[1]*op->bg[1] + a[2]*op->bg[2] - b;
        double Y[16];
        ox_sh_basis(sh_deg, d, Y);
        /* dL/dc_l per Gaussian of this ray: sparse map over the tape's Gaussians */
        int64_t ncap = tape.nG > 0 ? tape.nG : 1;
        int64_t* ids = malloc((size_t)ncap * sizeof(int64_t));
        double (*dcl)[3] = calloc((size_t)ncap, sizeof *dcl);
        int64_t nid = 0;
        double Cle[3] = {0, 0, 0};
        for (int64_t si = 0; si < tape.nS; si++) {
            ox_sample* s = &tape.S[si];
            double e = exp(-s->sigma * s->dtk);
            double alpha = 1.0 - e, Tn = s->T * e, w = s->T * alpha;
            for (int c = 0; c < 3; c++) Cle[c] += w * s->c[c];
            double dsig = 0;
            for (int c = 0; c < 3; c++) dsig += a[c] * (Tn * s->c[c] - (r.C[c] - Cle[c]));
            dsig = s->dtk * (dsig - dTf * r.T);
            double dci[3] = { a[0]*w, a[1]*w, a[2]*w };
            for (int64_t gi = s->first; gi < s->first + s->count; gi++) {
                ox_contrib* cb = &tape.G[gi];
                const ox_prim* pr = &P[cb->l];
                double pre[3], cl[3];
                prim_colour(pr, Y, d, cl, pre);
                double dg = dsig;
                for (int c = 0; c < 3; c++) dg += dci[c] * (cl[c] - s->c[c]) / s->sigma;
                /* dc_l accumulation (linear search is fine for an oracle) */
                int64_t slot = -1;
                for (int64_t q = nid - 1; q >= 0; q--) if (ids[q] == cb->l) { slot = q; break; }
                if (slot < 0) { slot = nid++; ids[slot] = cb->l; }
                for (int c = 0; c < 3; c++) dcl[slot][c] += dci[c] * cb->g / s->sigma;
                /* geometry */
                double x[3] = { o[0] + cb->t*d[0], o[1] + cb->t*d[1], o[2] + cb->t*d[2] };
                double xm[3] = { x[0]-pr->mu[0], x[1]-pr->mu[1], x[2]-pr->mu[2] };
                double y[3];
                for (int j = 0; j < 3; j++) y[j] = pr->M[3*j]*xm[0] + pr->M[3*j+1]*xm[1] + pr->M[3*j+2]*xm[2];
                double wg = dg * cb->g;
                atomic_add(&g_dens[cb->l], wg / pr->sig);
                for (int k = 0; k < 3; k++) {
                    double v = pr->M[k]*y[0] + pr->M[3+k]*y[1] + pr->M[6+k]*y[2];   /* (M^T y)_k */
                    atomic_add(&g_means[3*cb->l + k], wg * v);
                }
                for (int j = 0; j < 3; j++)
                    for (int k = 0; k < 3; k++)
                        atomic_add(&gM[9*cb->l + 3*j + k], -wg * y[j] * xm[k]);
            }
        }
        for (int64_t q = 0; q < nid; q++) {
            const ox_prim* pr = &P[ids[q]];
            double pre[3], cl[3];
            prim_colour(pr, Y, d, cl, pre);
            for (int k = 0; k < nk; k++)
                for (int c = 0; c < 3; c++)
                    if (pre[c] > 0) atomic_add(&g_sh[((int64_t)ids[q]*nk + k)*3 + c], Y[k] * dcl[q][c]);
            /* lobe j: dc/da_c = e_j; dc_c/dlambda = a_c e_j (mu.d - 1); dc_c/dmu = a_c e_j lambda d;
             * mu = u/|u| gives du = (dmu - mu (mu.dmu)) / |u| */
            for (int j = 0; j < pr->nsg; j++) {
                const double* rj = pr->sg + 7*j;
                double cosv, e = sg_lobe(pr, j, d, &cosv);
                double m[3], sa = 0;
                for (int c = 0; c < 3; c++) { m[c] = pre[c] > 0 ? dcl[q][c] : 0.0; sa += m[c] * rj[4 + c]; }
                double* gj = g_sg + ((int64_t)ids[q]*pr->nsg + j)*7;
                for (int c = 0; c < 3; c++) atomic_add(&gj[4 + c], m[c] * e);
                atomic_add(&gj[3], sa * e * (cosv - 1.0));
                double nu = sqrt(rj[0]*rj[0] + rj[1]*rj[1] + rj[2]*rj[2]);
                double mu[3] = { rj[0]/nu, rj[1]/nu, rj[2]/nu };
                double dmu[3] = { sa*e*rj[3]*d[0], sa*e*rj[3]*d[1], sa*e*rj[3]*d[2] };
                double md = mu[0]*dmu[0] + mu[1]*dmu[1] + mu[2]*dmu[2];
                for (int c = 0; c < 3; c++) atomic_add(&gj[c], (dmu[c] - mu[c]*md) / nu);
            }
        }
        free(ids); free(dcl); free(tape.S); free(tape.G);
    }

    /* chain dL/dM to scales and quaternions */
    #pragma omp parallel for schedule(static)
    for (int64_t l = 0; l < n; l++) {
        const ox_prim* pr = &P[l];
        const double* G = gM + 9*l;
        double dR[9] = {0};
        for (int j = 0; j < 3; j++) {
            double ds = 0;
            for (int k = 0; k < 3; k++) {
                /* M_jk = R_kj / s_j */
                ds += G[3*j + k] * (-pr->R[3*k + j] / (pr->s[j] * pr->s[j]));
                dR[3*k + j] += G[3*j + k] / pr->s[j];
            }
            g_scales[3*l + j] += ds;
        }
        const double* q = quats + 4*l;
        double nq = sqrt(q[0]*q[0] + q[1]*q[1] + q[2]*q[2] + q[3]*q[3]);
        double w = q[0]/nq, x = q[1]/nq, y = q[2]/nq, z = q[3]/nq;
        /* partial derivatives of R(w,x,y,z) entries */
        double dw = dR[1]*(-2*z) + dR[2]*(2*y) + dR[3]*(2*z) + dR[5]*(-2*x) + dR[6]*(-2*y) + dR[7]*(2*x);
        double dx = dR[1]*(2*y) + dR[2]*(2*z) + dR[3]*(2*y) + dR[4]*(-4*x) + dR[5]*(-2*w)
                  + dR[6]*(2*z) + dR[7]*(2*w) + dR[8]*(-4*x);
        double dy = dR[0]*(-4*y) + dR[1]*(2*x) + dR[2]*(2*w) + dR[3]*(2*x) + dR[5]*(2*z)
                  + dR[6]*(-2*w) + dR[7]*(2*z) + dR[8]*(-4*y);
        double dz = dR[0]*(-4*z) + dR[1]*(-2*w) + dR[2]*(2*x) + dR[3]*(2*w) + dR[4]*(-4*z)
                  + dR[5]*(2*y) + dR[6]*(2*x) + dR[7]*(2*y);
        double dot = w*dw + x*dx + y*dy + z*dz;
        g_quats[4*l + 0] += (dw - w*dot) / nq;
        g_quats[4*l + 1] += (dx - x*dot) / nq;
        g_quats[4*l + 2] += (dy - y*dot) / nq;
        g_quats[4*l + 3] += (dz - z*dot) / nq;
    }
    free(gM); free(P);
    return nerr;
}

/* Ray (origin, unit direction) of a pixel -- exposed for tests. */
void ox_ray(const ox_camera* cam, int64_t pix, double* o, double* d) { make_ray(cam, pix, o, d); }

/* Chords of a ray against every Gaussian -- exposed for tests.  tin/tout are
 * NaN where the chord is empty. */
void ox_chords(int64_t n, const double* means, const double* scales, const double* quats,
               const double* dens, double sigma_eps, const double* o, const double* d,
               double* tin, double* tout)
{
    for (int64_t l = 0; l < n; l++) {
        ox_prim p;
        prim_setup(&p, means + 3*l, scales + 3*l, quats + 4*l, dens[l], NULL, 0, sigma_eps);
        double a, b;
        if (chord(&p, o, d, &a, &b)) { tin[l] = a; tout[l] = b; }
        else { tin[l] = NAN; tout[l] = NAN; }
    }
}
