/* FP64 CPU oracle of the learned reconstruction network (test infrastructure).
 *
 * TEST INFRASTRUCTURE ONLY: only the tests and the smoke check load it. It
 * shares no code with the CUDA path. Direct loops, no blocking or fusion:
 *   conv3x3 (zero padding) + bias (+ ReLU), 2x2 average pool, nearest 2x
 *   upsample, channel concatenation, pixel shuffle (head channel
 *   k = 4 c + 2 dy + dx -> channel c of full-resolution pixel (2y+dy, 2x+dx)),
 *   bilinear 2x upsample with half-pixel centres and clamping, MSE.
 * Backward passes are derived by hand from those definitions; the tests check
 * them against central finite differences.
 *
 * Network (h x w half resolution; channels in brackets):
 *   e1 = relu(c1b(relu(c1a(in[4 + 12 zero])))) [32]
 *   e2 = relu(c2b(relu(c2a(pool(e1))))) [64]
 *   b  = relu(c3b(relu(c3a(pool(e2))))) [128]
 *   d2 = relu(d2b(relu(d2a(concat(up(b), e2))))) [64]
 *   d1 = relu(d1b(relu(d1a(concat(up(d2), e1))))) [32]
 *   out = bilinear_2x(in) + shuffle(head(d1)) [4 at 2h x 2w]
 * Parameters, in order, per layer: W[Cout][9][Cin] (tap = 3 (dy+1) + (dx+1)),
 * then b[Cout]; layers c1a c1b c2a c2b c3a c3b d2a d2b d1a d1b head.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NL 11
static const int CIN[NL] = {16, 32, 32, 64, 64, 128, 192, 64, 96, 32, 32};
static const int COUT[NL] = {32, 32, 64, 64, 128, 128, 64, 64, 32, 32, 16};

int64_t ou_param_count(void) {
  int64_t n = 0;
  for (int L = 0; L < NL; ++L) n += (int64_t)COUT[L] * 9 * CIN[L] + COUT[L];
  return n;
}

static void offsets(int64_t* wo, int64_t* bo) {
  int64_t n = 0;
  for (int L = 0; L < NL; ++L) {
    wo[L] = n;
    n += (int64_t)COUT[L] * 9 * CIN[L];
    bo[L] = n;
    n += COUT[L];
  }
}

#define AT(t, n, y, x, c, H, W, C) (t)[((((int64_t)(n) * (H) + (y)) * (W) + (x)) * (C)) + (c)]

/* out[n,y,x,co] = b[co] + sum_{dy,dx,ci} in[n,y+dy,x+dx,ci] w[co][tap][ci] (zero outside) */
static void conv_fwd(const double* in, int N, int H, int W, int Cin, const double* w, const double* b, int Cout,
                     int relu, double* out) {
  for (int n = 0; n < N; ++n)
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x)
        for (int co = 0; co < Cout; ++co) {
          double s = b[co];
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int yy = y + dy, xx = x + dx;
              if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
              int tap = 3 * (dy + 1) + (dx + 1);
              const double* wr = w + ((int64_t)co * 9 + tap) * Cin;
              for (int ci = 0; ci < Cin; ++ci) s += AT(in, n, yy, xx, ci, H, W, Cin) * wr[ci];
            }
          AT(out, n, y, x, co, H, W, Cout) = (relu && s < 0.0) ? 0.0 : s;
        }
}

/* dz = gradient w.r.t. the pre-activation output; accumulates dw, db, din */
static void conv_bwd(const double* in, int N, int H, int W, int Cin, const double* w, int Cout, const double* dz,
                     double* dw, double* db, double* din) {
  for (int n = 0; n < N; ++n)
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x)
        for (int co = 0; co < Cout; ++co) {
          double g = AT(dz, n, y, x, co, H, W, Cout);
          if (g == 0.0) continue;
          db[co] += g;
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int yy = y + dy, xx = x + dx;
              if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
              int tap = 3 * (dy + 1) + (dx + 1);
              for (int ci = 0; ci < Cin; ++ci) {
                dw[((int64_t)co * 9 + tap) * Cin + ci] += g * AT(in, n, yy, xx, ci, H, W, Cin);
                if (din) AT(din, n, yy, xx, ci, H, W, Cin) += g * w[((int64_t)co * 9 + tap) * Cin + ci];
              }
            }
        }
}

static void pool_fwd(const double* in, int N, int H, int W, int C, double* out) {
  for (int n = 0; n < N; ++n)
    for (int y = 0; y < H / 2; ++y)
      for (int x = 0; x < W / 2; ++x)
        for (int c = 0; c < C; ++c)
          AT(out, n, y, x, c, H / 2, W / 2, C) =
              0.25 * (AT(in, n, 2 * y, 2 * x, c, H, W, C) + AT(in, n, 2 * y, 2 * x + 1, c, H, W, C) +
                      AT(in, n, 2 * y + 1, 2 * x, c, H, W, C) + AT(in, n, 2 * y + 1, 2 * x + 1, c, H, W, C));
}
static void pool_bwd(const double* dout, int N, int H, int W, int C, double* din) {
  for (int n = 0; n < N; ++n)
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x)
        for (int c = 0; c < C; ++c) AT(din, n, y, x, c, H, W, C) += 0.25 * AT(dout, n, y / 2, x / 2, c, H / 2, W / 2, C);
}
/* nearest 2x: out (2H x 2W) from in (H x W) */
static void up_fwd(const double* in, int N, int H, int W, int C, double* out) {
  for (int n = 0; n < N; ++n)
    for (int y = 0; y < 2 * H; ++y)
      for (int x = 0; x < 2 * W; ++x)
        for (int c = 0; c < C; ++c) AT(out, n, y, x, c, 2 * H, 2 * W, C) = AT(in, n, y / 2, x / 2, c, H, W, C);
}
static void up_bwd(const double* dout, int N, int H, int W, int C, double* din) {
  for (int n = 0; n < N; ++n)
    for (int y = 0; y < 2 * H; ++y)
      for (int x = 0; x < 2 * W; ++x)
        for (int c = 0; c < C; ++c) AT(din, n, y / 2, x / 2, c, H, W, C) += AT(dout, n, y, x, c, 2 * H, 2 * W, C);
}
static void concat(const double* a, int Ca, const double* b, int Cb, int64_t P, double* out) {
  for (int64_t p = 0; p < P; ++p) {
    for (int c = 0; c < Ca; ++c) out[p * (Ca + Cb) + c] = a[p * Ca + c];
    for (int c = 0; c < Cb; ++c) out[p * (Ca + Cb) + Ca + c] = b[p * Cb + c];
  }
}
static void split_add(const double* g, int Ca, int Cb, int64_t P, double* ga, double* gb) {
  for (int64_t p = 0; p < P; ++p) {
    for (int c = 0; c < Ca; ++c) ga[p * Ca + c] += g[p * (Ca + Cb) + c];
    for (int c = 0; c < Cb; ++c) gb[p * Cb + c] += g[p * (Ca + Cb) + Ca + c];
  }
}
/* bilinear 2x with half-pixel centres: full pixel X samples half-res coordinate
 * X/2 - 1/4; neighbours clamped to the image */
void ou_bilinear2x(const double* in, int N, int h, int w, int C, double* out) {
  for (int n = 0; n < N; ++n)
    for (int Y = 0; Y < 2 * h; ++Y)
      for (int X = 0; X < 2 * w; ++X) {
        double ux = 0.5 * X - 0.25, uy = 0.5 * Y - 0.25;
        int x0 = (int)floor(ux), y0 = (int)floor(uy);
        double fx = ux - x0, fy = uy - y0;
        int xa = x0 < 0 ? 0 : (x0 > w - 1 ? w - 1 : x0), xb = x0 + 1 > w - 1 ? w - 1 : (x0 + 1 < 0 ? 0 : x0 + 1);
        int ya = y0 < 0 ? 0 : (y0 > h - 1 ? h - 1 : y0), yb = y0 + 1 > h - 1 ? h - 1 : (y0 + 1 < 0 ? 0 : y0 + 1);
        for (int c = 0; c < C; ++c)
          AT(out, n, Y, X, c, 2 * h, 2 * w, C) =
              (1 - fy) * ((1 - fx) * AT(in, n, ya, xa, c, h, w, C) + fx * AT(in, n, ya, xb, c, h, w, C)) +
              fy * ((1 - fx) * AT(in, n, yb, xa, c, h, w, C) + fx * AT(in, n, yb, xb, c, h, w, C));
      }
}

typedef struct {
  double *in16, *a1, *e1, *p1, *a2, *e2, *p2, *a3, *b3, *ub, *cat2, *a4, *d2, *ud, *cat1, *a5, *d1, *head;
} acts;

static double* z(int64_t n) { return (double*)calloc(n > 0 ? n : 1, sizeof(double)); }

static void acts_free(acts* A) {
  double** p = (double**)A;
  for (size_t i = 0; i < sizeof(acts) / sizeof(double*); ++i) free(p[i]);
}

static void forward(const double* prm, const double* in, int N, int h, int w, acts* A, double* out) {
  int64_t wo[NL], bo[NL];
  offsets(wo, bo);
  const int64_t P1 = (int64_t)N * h * w, P2 = P1 / 4, P3 = P1 / 16;
  A->in16 = z(P1 * 16);
  for (int64_t p = 0; p < P1; ++p)
    for (int c = 0; c < 4; ++c) A->in16[p * 16 + c] = in[p * 4 + c];
  A->a1 = z(P1 * 32); A->e1 = z(P1 * 32); A->p1 = z(P2 * 32); A->a2 = z(P2 * 64); A->e2 = z(P2 * 64);
  A->p2 = z(P3 * 64); A->a3 = z(P3 * 128); A->b3 = z(P3 * 128); A->ub = z(P2 * 128); A->cat2 = z(P2 * 192);
  A->a4 = z(P2 * 64); A->d2 = z(P2 * 64); A->ud = z(P1 * 64); A->cat1 = z(P1 * 96); A->a5 = z(P1 * 32);
  A->d1 = z(P1 * 32); A->head = z(P1 * 16);
  conv_fwd(A->in16, N, h, w, 16, prm + wo[0], prm + bo[0], 32, 1, A->a1);
  conv_fwd(A->a1, N, h, w, 32, prm + wo[1], prm + bo[1], 32, 1, A->e1);
  pool_fwd(A->e1, N, h, w, 32, A->p1);
  conv_fwd(A->p1, N, h / 2, w / 2, 32, prm + wo[2], prm + bo[2], 64, 1, A->a2);
  conv_fwd(A->a2, N, h / 2, w / 2, 64, prm + wo[3], prm + bo[3], 64, 1, A->e2);
  pool_fwd(A->e2, N, h / 2, w / 2, 64, A->p2);
  conv_fwd(A->p2, N, h / 4, w / 4, 64, prm + wo[4], prm + bo[4], 128, 1, A->a3);
  conv_fwd(A->a3, N, h / 4, w / 4, 128, prm + wo[5], prm + bo[5], 128, 1, A->b3);
  up_fwd(A->b3, N, h / 4, w / 4, 128, A->ub);
  concat(A->ub, 128, A->e2, 64, P2, A->cat2);
  conv_fwd(A->cat2, N, h / 2, w / 2, 192, prm + wo[6], prm + bo[6], 64, 1, A->a4);
  conv_fwd(A->a4, N, h / 2, w / 2, 64, prm + wo[7], prm + bo[7], 64, 1, A->d2);
  up_fwd(A->d2, N, h / 2, w / 2, 64, A->ud);
  concat(A->ud, 64, A->e1, 32, P1, A->cat1);
  conv_fwd(A->cat1, N, h, w, 96, prm + wo[8], prm + bo[8], 32, 1, A->a5);
  conv_fwd(A->a5, N, h, w, 32, prm + wo[9], prm + bo[9], 32, 1, A->d1);
  conv_fwd(A->d1, N, h, w, 32, prm + wo[10], prm + bo[10], 16, 0, A->head);
  ou_bilinear2x(in, N, h, w, 4, out);
  for (int n = 0; n < N; ++n)
    for (int Y = 0; Y < 2 * h; ++Y)
      for (int X = 0; X < 2 * w; ++X)
        for (int c = 0; c < 4; ++c)
          AT(out, n, Y, X, c, 2 * h, 2 * w, 4) += AT(A->head, n, Y / 2, X / 2, 4 * c + 2 * (Y & 1) + (X & 1), h, w, 16);
}

/* out: N x 2h x 2w x 4 */
void ou_forward(const double* prm, const double* in, int N, int h, int w, double* out) {
  acts A;
  memset(&A, 0, sizeof A);
  forward(prm, in, N, h, w, &A, out);
  acts_free(&A);
}

static void relu_mask(double* g, const double* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!(y[i] > 0.0)) g[i] = 0.0;
}

/* loss = mean over all outputs of (out - target)^2; grads (+= into zeroed) */
double ou_loss_grad(const double* prm, const double* in, const double* target, int N, int h, int w, double* out,
                    double* grad) {
  int64_t wo[NL], bo[NL];
  offsets(wo, bo);
  acts A;
  memset(&A, 0, sizeof A);
  forward(prm, in, N, h, w, &A, out);
  const int64_t P1 = (int64_t)N * h * w, P2 = P1 / 4, P3 = P1 / 16, cnt = P1 * 16;
  double loss = 0.0;
  double* gh = z(P1 * 16);
  for (int n = 0; n < N; ++n)
    for (int Y = 0; Y < 2 * h; ++Y)
      for (int X = 0; X < 2 * w; ++X)
        for (int c = 0; c < 4; ++c) {
          double d = AT(out, n, Y, X, c, 2 * h, 2 * w, 4) - AT(target, n, Y, X, c, 2 * h, 2 * w, 4);
          loss += d * d / (double)cnt;
          AT(gh, n, Y / 2, X / 2, 4 * c + 2 * (Y & 1) + (X & 1), h, w, 16) = 2.0 * d / (double)cnt;
        }
  memset(grad, 0, sizeof(double) * ou_param_count());
  double *g_d1 = z(P1 * 32), *g_a5 = z(P1 * 32), *g_cat1 = z(P1 * 96), *g_ud = z(P1 * 64), *g_e1 = z(P1 * 32);
  double *g_d2 = z(P2 * 64), *g_a4 = z(P2 * 64), *g_cat2 = z(P2 * 192), *g_ub = z(P2 * 128), *g_e2 = z(P2 * 64);
  double *g_b3 = z(P3 * 128), *g_a3 = z(P3 * 128), *g_p2 = z(P3 * 64), *g_a2 = z(P2 * 64), *g_p1 = z(P2 * 32);
  double *g_a1 = z(P1 * 32);
  conv_bwd(A.d1, N, h, w, 32, prm + wo[10], 16, gh, grad + wo[10], grad + bo[10], g_d1);
  relu_mask(g_d1, A.d1, P1 * 32);
  conv_bwd(A.a5, N, h, w, 32, prm + wo[9], 32, g_d1, grad + wo[9], grad + bo[9], g_a5);
  relu_mask(g_a5, A.a5, P1 * 32);
  conv_bwd(A.cat1, N, h, w, 96, prm + wo[8], 32, g_a5, grad + wo[8], grad + bo[8], g_cat1);
  split_add(g_cat1, 64, 32, P1, g_ud, g_e1);
  up_bwd(g_ud, N, h / 2, w / 2, 64, g_d2);
  relu_mask(g_d2, A.d2, P2 * 64);
  conv_bwd(A.a4, N, h / 2, w / 2, 64, prm + wo[7], 64, g_d2, grad + wo[7], grad + bo[7], g_a4);
  relu_mask(g_a4, A.a4, P2 * 64);
  conv_bwd(A.cat2, N, h / 2, w / 2, 192, prm + wo[6], 64, g_a4, grad + wo[6], grad + bo[6], g_cat2);
  split_add(g_cat2, 128, 64, P2, g_ub, g_e2);
  up_bwd(g_ub, N, h / 4, w / 4, 128, g_b3);
  relu_mask(g_b3, A.b3, P3 * 128);
  conv_bwd(A.a3, N, h / 4, w / 4, 128, prm + wo[5], 128, g_b3, grad + wo[5], grad + bo[5], g_a3);
  relu_mask(g_a3, A.a3, P3 * 128);
  conv_bwd(A.p2, N, h / 4, w / 4, 64, prm + wo[4], 128, g_a3, grad + wo[4], grad + bo[4], g_p2);
  pool_bwd(g_p2, N, h / 2, w / 2, 64, g_e2);
  relu_mask(g_e2, A.e2, P2 * 64);
  conv_bwd(A.a2, N, h / 2, w / 2, 64, prm + wo[3], 64, g_e2, grad + wo[3], grad + bo[3], g_a2);
  relu_mask(g_a2, A.a2, P2 * 64);
  conv_bwd(A.p1, N, h / 2, w / 2, 32, prm + wo[2], 64, g_a2, grad + wo[2], grad + bo[2], g_p1);
  pool_bwd(g_p1, N, h, w, 32, g_e1);
  relu_mask(g_e1, A.e1, P1 * 32);
  conv_bwd(A.a1, N, h, w, 32, prm + wo[1], 32, g_e1, grad + wo[1], grad + bo[1], g_a1);
  relu_mask(g_a1, A.a1, P1 * 32);
  conv_bwd(A.in16, N, h, w, 16, prm + wo[0], 32, g_a1, grad + wo[0], grad + bo[0], NULL);
  free(gh); free(g_d1); free(g_a5); free(g_cat1); free(g_ud); free(g_e1); free(g_d2); free(g_a4); free(g_cat2);
  free(g_ub); free(g_e2); free(g_b3); free(g_a3); free(g_p2); free(g_a2); free(g_p1); free(g_a1);
  acts_free(&A);
  return loss;
}

/* ==========================================================================
 * The BF16 network and the spread of an FP32-accumulating implementation.
 *
 * The learned path's definition fixes its precision: BF16 weights and
 * activations, FP32 accumulation. The functions below compute that network
 * in FP64 with the BF16 rounding points it implies: the RGBA input, every
 * convolution's output after bias and ReLU, every 2x2-pooled map and every
 * masked output gradient are rounded to BF16 (round to nearest even); the
 * head's output, the bilinear base and all other gradients stay unrounded.
 *
 * An implementation that rounds at the same points but accumulates in FP32
 * (in any order) differs from it through two effects, and alongside every
 * value the functions propagate sigma, the standard deviation of that
 * difference under the usual model of rounding errors as independent and
 * zero-mean:
 *   - accumulation: a sum of terms t_k carried in FP32 along a chain of at
 *     most `chain` sequential additions (each off by at most 2^-23 of the
 *     running sum, truncating adders included) has sigma <= 2^-23
 *     sqrt(chain) sum|t_k|; inputs with sigmas s_k add sum (w_k s_k)^2;
 *   - rounding flips: where the implementation's value before rounding is
 *     v + d, d ~ N(0, sigma^2), rnd(v + d) differs from rnd(v) by one BF16
 *     step only when v + d crosses the rounding boundary next to v: with
 *     probability Phi(-gap / sigma), computed per element from the oracle's
 *     own gap; so sigma after rounding is a step times the root of that
 *     probability, 0 for most elements;
 *   - ReLU passes sigma where its input is positive; where it clamps at
 *     s <= 0 the implementation's value is (s + d)_+, of mean square
 *     (s^2 + sigma^2) Phi(s / sigma) + s sigma phi(s / sigma);
 *   - a ReLU mask taken from a stored activation flips with the probability
 *     that the implementation's pre-activation has the other sign; the
 *     masked gradient then changes by the whole gradient.
 * A test then accepts |impl - oracle| <= k sigma elementwise (k = 8 in the
 * tests: under the model, far beyond any sample they take).
 * ======================================================================== */

/* round to the nearest BF16 value (8 significant bits), ties to even */
double ou_bf16(double v) {
  if (v == 0.0 || !isfinite(v)) return v;
  int e;
  frexp(v, &e); /* |v| = f 2^e, 0.5 <= f < 1 */
  int q = e - 8;
  if (q < -133) q = -133; /* BF16 subnormals: multiples of 2^-133 */
  double s = ldexp(v, -q);
  return ldexp(nearbyint(s), q);
}

/* the BF16 neighbours of a BF16 value r: one step up and one step down */
static void bf16_neighbours(double r, double* up, double* dn) {
  if (r == 0.0) {
    *up = ldexp(1.0, -133);
    *dn = -ldexp(1.0, -133);
    return;
  }
  int e;
  double f = frexp(fabs(r), &e);
  int q = e - 8;
  if (q < -133) q = -133;
  double step_out = ldexp(1.0, q);
  /* at a power of two the step toward zero is half as large */
  double step_in = (f == 0.5 && q > -133) ? ldexp(1.0, q - 1) : step_out;
  if (r > 0.0) {
    *up = r + step_out;
    *dn = r - step_in;
  } else {
    *up = r + step_in;
    *dn = r - step_out;
  }
}

static double Phi(double z) { return 0.5 * erfc(-z / sqrt(2.0)); }

/* variance of rnd(v + d) - rnd(v), d ~ N(0, s^2); *r = rnd(v) */
static double round_var(double v, double s, double* r) {
  double rv = ou_bf16(v);
  *r = rv;
  if (s == 0.0) return 0.0;
  double up, dn;
  bf16_neighbours(rv, &up, &dn);
  double hu = up - rv, hd = rv - dn;
  if (s > 0.25 * (hu < hd ? hu : hd)) /* several steps: the spread plus rounding noise */
    return s * s + (hu * hu + hd * hd) / 24.0;
  double pu = Phi(-(0.5 * (rv + up) - v) / s), pd = Phi(-(v - 0.5 * (rv + dn)) / s);
  return pu * hu * hu + pd * hd * hd;
}

/* mean square of (s + d)_+ for s <= 0, d ~ N(0, sg^2): (s^2 + sg^2) Phi(z)
 * + s sg phi(z), z = s / sg. The two terms cancel as z falls; below z = -8
 * the value (under 1e-15 sg^2) is taken as 0, and rounding never makes it
 * negative. */
static double relu_clamped_ms(double s, double sg) {
  if (sg == 0.0) return 0.0;
  double z = s / sg;
  if (z < -8.0) return 0.0;
  double v = (s * s + sg * sg) * Phi(z) + s * sg * exp(-0.5 * z * z) / sqrt(2.0 * M_PI);
  return v > 0.0 ? v : 0.0;
}

#define U23 (1.0 / 8388608.0)  /* 2^-23: one FP32 operation, truncating or not */
#define U24 (1.0 / 16777216.0) /* 2^-24: representation of a value in FP32 */

/* conv forward of the BF16 network: out = rnd(relu(b + sum in w)) with its
 * sigma (sout) and the probability that the implementation's
 * pre-activation has the other sign (pflip, may be NULL); rnd = 0 leaves the
 * output in FP32 (the head) */
static void conv_fwd_q(const double* in, const double* sin, int N, int H, int W, int Cin, const double* w,
                       const double* b, int Cout, int relu, int rnd, double* out, double* sout, double* pflip) {
  const double chain = 9.0 * Cin / 16.0 + 20.0;
  for (int n = 0; n < N; ++n)
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x)
        for (int co = 0; co < Cout; ++co) {
          double s = b[co], m = fabs(b[co]), var = 0.0;
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int yy = y + dy, xx = x + dx;
              if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
              int tap = 3 * (dy + 1) + (dx + 1);
              const double* wr = w + ((int64_t)co * 9 + tap) * Cin;
              for (int ci = 0; ci < Cin; ++ci) {
                double a = AT(in, n, yy, xx, ci, H, W, Cin), sa = AT(sin, n, yy, xx, ci, H, W, Cin);
                s += a * wr[ci];
                m += fabs(a * wr[ci]);
                var += wr[ci] * wr[ci] * sa * sa;
              }
            }
          const double sacc = U23 * sqrt(chain) * m + U24 * fabs(s);
          const double sg = sqrt(var + sacc * sacc);
          int64_t o = (((int64_t)n * H + y) * W + x) * Cout + co;
          if (pflip) pflip[o] = sg > 0.0 ? Phi(-fabs(s) / sg) : 0.0;
          if (relu && s <= 0.0) {
            out[o] = 0.0;
            sout[o] = sqrt(relu_clamped_ms(s, sg));
          } else if (rnd) {
            sout[o] = sqrt(round_var(s, sg, &out[o]));
          } else {
            out[o] = s;
            sout[o] = sg;
          }
        }
}

static void pool_fwd_q(const double* in, const double* sin, int N, int H, int W, int C, double* out, double* sout) {
  for (int n = 0; n < N; ++n)
    for (int y = 0; y < H / 2; ++y)
      for (int x = 0; x < W / 2; ++x)
        for (int c = 0; c < C; ++c) {
          double s = 0.0, m = 0.0, var = 0.0;
          for (int k = 0; k < 4; ++k) {
            double a = AT(in, n, 2 * y + (k >> 1), 2 * x + (k & 1), c, H, W, C);
            double sa = AT(sin, n, 2 * y + (k >> 1), 2 * x + (k & 1), c, H, W, C);
            s += a;
            m += fabs(a);
            var += 0.0625 * sa * sa;
          }
          const double sacc = 0.25 * U23 * sqrt(3.0) * m;
          int64_t o = (((int64_t)n * (H / 2) + y) * (W / 2) + x) * C + c;
          sout[o] = sqrt(round_var(0.25 * s, sqrt(var + sacc * sacc), &out[o]));
        }
}

/* dz = rnd(dy mask(y > 0)) (y = NULL: no ReLU) with its sigma, from dy's
 * sigma sdy and the stored activation's sign-flip probability py */
static void masked_q(const double* dy, const double* sdy, const double* y, const double* py, int64_t n, double* dz,
                     double* sdz) {
  for (int64_t i = 0; i < n; ++i) {
    double g = dy[i], sg = sdy[i];
    double v = g, var = sg * sg;
    if (y) {
      const int on = y[i] > 0.0;
      const double p = py[i];
      if (!on) v = 0.0;
      /* kept with probability 1 - p (the sigma of dy), else the other
       * choice: the whole gradient */
      var = (on ? (1.0 - p) * sg * sg : p * sg * sg) + p * (g * g);
    }
    if (y && !(y[i] > 0.0)) {
      dz[i] = 0.0;
      sdz[i] = sqrt(var);
      continue;
    }
    sdz[i] = sqrt(round_var(v, sqrt(var), &dz[i]));
  }
}

/* conv backward of the BF16 network from the masked gradient dz (BF16):
 * dw += sum dz in, db += sum dz, din += sum dz w (FP32 sums). vw, vb, vdin
 * accumulate the variance from the inputs' sigmas; mw, mb, mdin the sums of
 * |terms| for the accumulation terms. */
static void conv_bwd_q(const double* in, const double* sin, int N, int H, int W, int Cin, const double* w, int Cout,
                       const double* dz, const double* sdz, double* dw, double* vw, double* mw, double* db,
                       double* vb, double* mb, double* din, double* vdin, double* mdin) {
  for (int n = 0; n < N; ++n)
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x)
        for (int co = 0; co < Cout; ++co) {
          double g = AT(dz, n, y, x, co, H, W, Cout), sg = AT(sdz, n, y, x, co, H, W, Cout);
          if (g == 0.0 && sg == 0.0) continue;
          db[co] += g;
          vb[co] += sg * sg;
          mb[co] += fabs(g);
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int yy = y + dy, xx = x + dx;
              if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
              int tap = 3 * (dy + 1) + (dx + 1);
              for (int ci = 0; ci < Cin; ++ci) {
                int64_t k = ((int64_t)co * 9 + tap) * Cin + ci;
                double a = AT(in, n, yy, xx, ci, H, W, Cin), sa = AT(sin, n, yy, xx, ci, H, W, Cin);
                dw[k] += g * a;
                vw[k] += sg * sg * a * a + g * g * sa * sa;
                mw[k] += fabs(g * a);
                if (din) {
                  int64_t q = (((int64_t)n * H + yy) * W + xx) * Cin + ci;
                  din[q] += g * w[k];
                  vdin[q] += sg * sg * w[k] * w[k];
                  mdin[q] += fabs(g * w[k]);
                }
              }
            }
        }
}

/* turns accumulated variances v (in place) into sigmas with the
 * accumulation term of a chain of `chain` FP32 additions */
static void finish_sigma(const double* val, double* v, double* m, int64_t n, double chain) {
  for (int64_t i = 0; i < n; ++i) {
    const double sacc = U23 * sqrt(chain) * m[i] + U24 * fabs(val[i]);
    v[i] = sqrt(v[i] + sacc * sacc);
    m[i] = 0.0;
  }
}

typedef struct {
  double *in16, *a1, *e1, *p1, *a2, *e2, *p2, *a3, *b3, *ub, *cat2, *a4, *d2, *ud, *cat1, *a5, *d1, *head;
} qacts;

static void qacts_alloc(qacts* T, int64_t P1) {
  const int64_t P2 = P1 / 4, P3 = P1 / 16;
  T->in16 = z(P1 * 16); T->a1 = z(P1 * 32); T->e1 = z(P1 * 32); T->p1 = z(P2 * 32); T->a2 = z(P2 * 64);
  T->e2 = z(P2 * 64); T->p2 = z(P3 * 64); T->a3 = z(P3 * 128); T->b3 = z(P3 * 128); T->ub = z(P2 * 128);
  T->cat2 = z(P2 * 192); T->a4 = z(P2 * 64); T->d2 = z(P2 * 64); T->ud = z(P1 * 64); T->cat1 = z(P1 * 96);
  T->a5 = z(P1 * 32); T->d1 = z(P1 * 32); T->head = z(P1 * 16);
}

static void qacts_free(qacts* A) {
  double** p = (double**)A;
  for (size_t i = 0; i < sizeof(qacts) / sizeof(double*); ++i) free(p[i]);
}

/* the BF16 network's forward: values A, sigmas S, sign-flip probabilities F
 * of the ReLU outputs (F's entries for a1 e1 a2 e2 a3 b3 a4 d2 a5 d1) */
static void forward_q(const double* prm, const double* in, int N, int h, int w, qacts* A, qacts* S, qacts* F,
                      double* out, double* sout) {
  int64_t wo[NL], bo[NL];
  offsets(wo, bo);
  const int64_t P1 = (int64_t)N * h * w, P2 = P1 / 4;
  qacts_alloc(A, P1);
  qacts_alloc(S, P1);
  qacts_alloc(F, P1);
  /* the input is given in FP32; its BF16 copy feeds the first convolution */
  for (int64_t p = 0; p < P1; ++p)
    for (int c = 0; c < 4; ++c) A->in16[p * 16 + c] = ou_bf16(in[p * 4 + c]);
  conv_fwd_q(A->in16, S->in16, N, h, w, 16, prm + wo[0], prm + bo[0], 32, 1, 1, A->a1, S->a1, F->a1);
  conv_fwd_q(A->a1, S->a1, N, h, w, 32, prm + wo[1], prm + bo[1], 32, 1, 1, A->e1, S->e1, F->e1);
  pool_fwd_q(A->e1, S->e1, N, h, w, 32, A->p1, S->p1);
  conv_fwd_q(A->p1, S->p1, N, h / 2, w / 2, 32, prm + wo[2], prm + bo[2], 64, 1, 1, A->a2, S->a2, F->a2);
  conv_fwd_q(A->a2, S->a2, N, h / 2, w / 2, 64, prm + wo[3], prm + bo[3], 64, 1, 1, A->e2, S->e2, F->e2);
  pool_fwd_q(A->e2, S->e2, N, h / 2, w / 2, 64, A->p2, S->p2);
  conv_fwd_q(A->p2, S->p2, N, h / 4, w / 4, 64, prm + wo[4], prm + bo[4], 128, 1, 1, A->a3, S->a3, F->a3);
  conv_fwd_q(A->a3, S->a3, N, h / 4, w / 4, 128, prm + wo[5], prm + bo[5], 128, 1, 1, A->b3, S->b3, F->b3);
  qacts* T[2] = {A, S};
  for (int k = 0; k < 2; ++k) {
    up_fwd(T[k]->b3, N, h / 4, w / 4, 128, T[k]->ub);
    concat(T[k]->ub, 128, T[k]->e2, 64, P2, T[k]->cat2);
  }
  conv_fwd_q(A->cat2, S->cat2, N, h / 2, w / 2, 192, prm + wo[6], prm + bo[6], 64, 1, 1, A->a4, S->a4, F->a4);
  conv_fwd_q(A->a4, S->a4, N, h / 2, w / 2, 64, prm + wo[7], prm + bo[7], 64, 1, 1, A->d2, S->d2, F->d2);
  for (int k = 0; k < 2; ++k) {
    up_fwd(T[k]->d2, N, h / 2, w / 2, 64, T[k]->ud);
    concat(T[k]->ud, 64, T[k]->e1, 32, P1, T[k]->cat1);
  }
  conv_fwd_q(A->cat1, S->cat1, N, h, w, 96, prm + wo[8], prm + bo[8], 32, 1, 1, A->a5, S->a5, F->a5);
  conv_fwd_q(A->a5, S->a5, N, h, w, 32, prm + wo[9], prm + bo[9], 32, 1, 1, A->d1, S->d1, F->d1);
  conv_fwd_q(A->d1, S->d1, N, h, w, 32, prm + wo[10], prm + bo[10], 16, 0, 0, A->head, S->head, NULL);
  /* out = bilinear 2x of the FP32 input + the shuffled head, in FP32 */
  ou_bilinear2x(in, N, h, w, 4, out);
  double* absin = z(P1 * 4);
  for (int64_t i = 0; i < P1 * 4; ++i) absin[i] = fabs(in[i]);
  ou_bilinear2x(absin, N, h, w, 4, sout); /* sum of |terms| of the bilinear blend */
  free(absin);
  for (int n = 0; n < N; ++n)
    for (int Y = 0; Y < 2 * h; ++Y)
      for (int X = 0; X < 2 * w; ++X)
        for (int c = 0; c < 4; ++c) {
          int k = 4 * c + 2 * (Y & 1) + (X & 1);
          double hv = AT(A->head, n, Y / 2, X / 2, k, h, w, 16), hs = AT(S->head, n, Y / 2, X / 2, k, h, w, 16);
          double* o = &AT(out, n, Y, X, c, 2 * h, 2 * w, 4);
          double* so = &AT(sout, n, Y, X, c, 2 * h, 2 * w, 4);
          *o += hv;
          const double sacc = U23 * sqrt(8.0) * (*so + fabs(hv)) + U24 * fabs(*o);
          *so = sqrt(hs * hs + sacc * sacc);
        }
}

/* out and its sigma sout: N x 2h x 2w x 4 */
void ou_bf16_forward(const double* prm, const double* in, int N, int h, int w, double* out, double* sout) {
  qacts A, S, F;
  memset(&A, 0, sizeof A);
  memset(&S, 0, sizeof S);
  memset(&F, 0, sizeof F);
  forward_q(prm, in, N, h, w, &A, &S, &F, out, sout);
  qacts_free(&A);
  qacts_free(&S);
  qacts_free(&F);
}

/* Loss, gradients and output of the BF16 network with the sigma of every
 * output value (sout) and every gradient (sgrad). prm holds the weights the
 * implementation multiplies with (BF16 values) and FP32 biases; in and
 * target hold FP32 values. */
double ou_bf16_loss_grad(const double* prm, const double* in, const double* target, int N, int h, int w,
                         double* out, double* sout, double* grad, double* sgrad) {
  int64_t wo[NL], bo[NL];
  offsets(wo, bo);
  qacts A, S, F;
  memset(&A, 0, sizeof A);
  memset(&S, 0, sizeof S);
  memset(&F, 0, sizeof F);
  forward_q(prm, in, N, h, w, &A, &S, &F, out, sout);
  const int64_t P1 = (int64_t)N * h * w, P2 = P1 / 4, P3 = P1 / 16, cnt = P1 * 16;
  const int64_t np = ou_param_count();
  double loss = 0.0;
  double *gh = z(P1 * 16), *sgh = z(P1 * 16);
  for (int n = 0; n < N; ++n)
    for (int Y = 0; Y < 2 * h; ++Y)
      for (int X = 0; X < 2 * w; ++X)
        for (int c = 0; c < 4; ++c) {
          double d = AT(out, n, Y, X, c, 2 * h, 2 * w, 4) - AT(target, n, Y, X, c, 2 * h, 2 * w, 4);
          double sd = AT(sout, n, Y, X, c, 2 * h, 2 * w, 4);
          loss += d * d / (double)cnt;
          int k = 4 * c + 2 * (Y & 1) + (X & 1);
          double gv = 2.0 * d / (double)cnt;
          AT(gh, n, Y / 2, X / 2, k, h, w, 16) = gv;
          /* d out = 2 (out - target) scale, scale = 1/count in FP32 */
          double sr = 2.0 * sd / (double)cnt, sa = 3.0 * U24 * fabs(gv);
          AT(sgh, n, Y / 2, X / 2, k, h, w, 16) = sqrt(sr * sr + sa * sa);
        }
  memset(grad, 0, sizeof(double) * np);
  memset(sgrad, 0, sizeof(double) * np);
  double* mg = z(np);
  /* gradient buffers (values g_*, variances then sigmas v_*, sums of |terms| m_*) */
#define GB(name, n) double *g_##name = z(n), *v_##name = z(n), *m_##name = z(n)
  GB(d1, P1 * 32); GB(a5, P1 * 32); GB(cat1, P1 * 96); GB(d2, P2 * 64); GB(a4, P2 * 64); GB(cat2, P2 * 192);
  GB(b3, P3 * 128); GB(a3, P3 * 128); GB(p2, P3 * 64); GB(a2, P2 * 64); GB(p1, P2 * 32); GB(a1, P1 * 32);
#undef GB
  double *dz = z(P1 * 96), *sdz = z(P1 * 96);
  const double Pw[3] = {(double)P1, (double)P2, (double)P3};
  /* one layer: masked gradient from (gy, sy) of the output (yv, fy: the
   * stored activation and its sign-flip probabilities; NULL for the head),
   * weight/bias gradients, input gradient into (gi, vi, mi) */
#define LAYER(L, gy, sy, yv, fy, C, lvl, x, xs, Cin, Hh, Ww, gi, vi, mi)                                       \
  do {                                                                                                        \
    masked_q(gy, sy, yv, fy, (int64_t)(Pw[lvl] * (C)), dz, sdz);                                             \
    conv_bwd_q(x, xs, N, Hh, Ww, Cin, prm + wo[L], C, dz, sdz, grad + wo[L], sgrad + wo[L], mg + wo[L],    \
               grad + bo[L], sgrad + bo[L], mg + bo[L], gi, vi, mi);                                         \
    finish_sigma(grad + wo[L], sgrad + wo[L], mg + wo[L], (int64_t)(C) * 9 * (Cin), Pw[lvl] / 16.0 + 40.0); \
    finish_sigma(grad + bo[L], sgrad + bo[L], mg + bo[L], (C), Pw[lvl] / 16.0 + 40.0);                      \
    if (gi) finish_sigma(gi, vi, mi, (int64_t)(Pw[lvl] * (Cin)), 9.0 * (C) / 16.0 + 20.0);                   \
  } while (0)
  LAYER(10, gh, sgh, NULL, NULL, 16, 0, A.d1, S.d1, 32, h, w, g_d1, v_d1, m_d1);
  LAYER(9, g_d1, v_d1, A.d1, F.d1, 32, 0, A.a5, S.a5, 32, h, w, g_a5, v_a5, m_a5);
  LAYER(8, g_a5, v_a5, A.a5, F.a5, 32, 0, A.cat1, S.cat1, 96, h, w, g_cat1, v_cat1, m_cat1);
  /* nearest-upsampling gradient: g_d2 = sum of the 4 children of g_cat1[:, 0..64) (FP32) */
  for (int n = 0; n < N; ++n)
    for (int Y = 0; Y < h; ++Y)
      for (int X = 0; X < w; ++X)
        for (int c = 0; c < 64; ++c) {
          int64_t o = (((int64_t)n * (h / 2) + Y / 2) * (w / 2) + X / 2) * 64 + c;
          int64_t s = (((int64_t)n * h + Y) * w + X) * 96 + c;
          g_d2[o] += g_cat1[s];
          v_d2[o] += v_cat1[s] * v_cat1[s];
          m_d2[o] += fabs(g_cat1[s]);
        }
  finish_sigma(g_d2, v_d2, m_d2, P2 * 64, 4.0);
  LAYER(7, g_d2, v_d2, A.d2, F.d2, 64, 1, A.a4, S.a4, 64, h / 2, w / 2, g_a4, v_a4, m_a4);
  LAYER(6, g_a4, v_a4, A.a4, F.a4, 64, 1, A.cat2, S.cat2, 192, h / 2, w / 2, g_cat2, v_cat2, m_cat2);
  for (int n = 0; n < N; ++n)
    for (int Y = 0; Y < h / 2; ++Y)
      for (int X = 0; X < w / 2; ++X)
        for (int c = 0; c < 128; ++c) {
          int64_t o = (((int64_t)n * (h / 4) + Y / 2) * (w / 4) + X / 2) * 128 + c;
          int64_t s = (((int64_t)n * (h / 2) + Y) * (w / 2) + X) * 192 + c;
          g_b3[o] += g_cat2[s];
          v_b3[o] += v_cat2[s] * v_cat2[s];
          m_b3[o] += fabs(g_cat2[s]);
        }
  finish_sigma(g_b3, v_b3, m_b3, P3 * 128, 4.0);
  LAYER(5, g_b3, v_b3, A.b3, F.b3, 128, 2, A.a3, S.a3, 128, h / 4, w / 4, g_a3, v_a3, m_a3);
  LAYER(4, g_a3, v_a3, A.a3, F.a3, 128, 2, A.p2, S.p2, 64, h / 4, w / 4, g_p2, v_p2, m_p2);
  /* average-pooling gradient: e2's gradient (in cat2[:, 128..)) += g_p2 / 4 (FP32) */
  {
    double *ge2 = z(P2 * 64), *se2 = z(P2 * 64);
    for (int64_t p = 0; p < P2; ++p)
      for (int c = 0; c < 64; ++c) {
        int n = (int)(p / ((int64_t)(h / 2) * (w / 2))), r = (int)(p % ((int64_t)(h / 2) * (w / 2)));
        int Y = r / (w / 2), X = r % (w / 2);
        int64_t o = (((int64_t)n * (h / 4) + Y / 2) * (w / 4) + X / 2) * 64 + c;
        double a = g_cat2[p * 192 + 128 + c], b = 0.25 * g_p2[o], v = a + b;
        double sa = v_cat2[p * 192 + 128 + c], sb = 0.25 * v_p2[o], sacc = U24 * fabs(v);
        ge2[p * 64 + c] = v;
        se2[p * 64 + c] = sqrt(sa * sa + sb * sb + sacc * sacc);
      }
    LAYER(3, ge2, se2, A.e2, F.e2, 64, 1, A.a2, S.a2, 64, h / 2, w / 2, g_a2, v_a2, m_a2);
    free(ge2);
    free(se2);
  }
  LAYER(2, g_a2, v_a2, A.a2, F.a2, 64, 1, A.p1, S.p1, 32, h / 2, w / 2, g_p1, v_p1, m_p1);
  {
    double *ge1 = z(P1 * 32), *se1 = z(P1 * 32);
    for (int64_t p = 0; p < P1; ++p)
      for (int c = 0; c < 32; ++c) {
        int n = (int)(p / ((int64_t)h * w)), r = (int)(p % ((int64_t)h * w));
        int Y = r / w, X = r % w;
        int64_t o = (((int64_t)n * (h / 2) + Y / 2) * (w / 2) + X / 2) * 32 + c;
        double a = g_cat1[p * 96 + 64 + c], b = 0.25 * g_p1[o], v = a + b;
        double sa = v_cat1[p * 96 + 64 + c], sb = 0.25 * v_p1[o], sacc = U24 * fabs(v);
        ge1[p * 32 + c] = v;
        se1[p * 32 + c] = sqrt(sa * sa + sb * sb + sacc * sacc);
      }
    LAYER(1, ge1, se1, A.e1, F.e1, 32, 0, A.a1, S.a1, 32, h, w, g_a1, v_a1, m_a1);
    free(ge1);
    free(se1);
  }
  LAYER(0, g_a1, v_a1, A.a1, F.a1, 32, 0, A.in16, S.in16, 16, h, w, NULL, NULL, NULL);
#undef LAYER
  free(gh); free(sgh); free(mg); free(dz); free(sdz);
  double* bufs[] = {g_d1, v_d1, m_d1, g_a5, v_a5, m_a5, g_cat1, v_cat1, m_cat1, g_d2, v_d2, m_d2, g_a4, v_a4, m_a4,
                    g_cat2, v_cat2, m_cat2, g_b3, v_b3, m_b3, g_a3, v_a3, m_a3, g_p2, v_p2, m_p2, g_a2, v_a2, m_a2,
                    g_p1, v_p1, m_p1, g_a1, v_a1, m_a1};
  for (size_t i = 0; i < sizeof bufs / sizeof bufs[0]; ++i) free(bufs[i]);
  qacts_free(&A);
  qacts_free(&S);
  qacts_free(&F);
  return loss;
}
