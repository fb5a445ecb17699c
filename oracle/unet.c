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
