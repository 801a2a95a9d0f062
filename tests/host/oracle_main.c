/* Stand-alone driver of oracle/stokes_oracle.c for the sanitizer build (tests/test_sanitizers.py):
 * reads a case file, runs every entry point of the oracle on it (node sum with and without a
 * selection, free targets, Kress weights, the argument checks) and writes the results, so that
 * AddressSanitizer and UndefinedBehaviorSanitizer watch every path the tests use.
 * Usage: oracle_main <case.bin> <out.bin>
 * case.bin: int32 N, n_curves, n_sel, n_free; float64 period, mu, jump; int32 off[n_curves + 1],
 *           kind[n_curves]; float64 nodes[2N], weights[N], normals[2N], curvature[N],
 *           slp[2 n_slp], dlp[2 n_dlp]; int32 sel[n_sel]; float64 free[2 n_free].
 * out.bin:  float64 nodes_out[2N], sel_out[2 n_sel], free_out[2 n_free], R[n_0] (Kress weights
 *           of the first vesicle's size, when there is one); then int32 status codes of the
 *           deliberately bad calls. */
#include <stdio.h>
#include <stdlib.h>

int ora_sum(int, int, const int *, const int *, const double *, const double *, const double *,
            const double *, double, double, const double *, const double *, double, int,
            const int *, double *, int);
int ora_sum_free(int, int, const int *, const int *, const double *, const double *,
                 const double *, double, double, const double *, const double *, int,
                 const double *, double *, int);
int ora_kress_weights(int, double *);

static void *xmalloc(size_t n) {
    void *p = malloc(n ? n : 1);
    if (!p) exit(3);
    return p;
}

static void rd(void *p, size_t sz, size_t n, FILE *f) {
    if (n && fread(p, sz, n, f) != n) exit(4);
}

int main(int argc, char **argv) {
    if (argc < 3) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    int hdr[4];
    double par[3];
    rd(hdr, 4, 4, f);
    rd(par, 8, 3, f);
    const int N = hdr[0], nc = hdr[1], nsel = hdr[2], nfree = hdr[3];
    int *off = xmalloc(sizeof(int) * (nc + 1)), *kind = xmalloc(sizeof(int) * nc);
    rd(off, 4, nc + 1, f);
    rd(kind, 4, nc, f);
    int n_slp = 0, first_ves = 0;
    for (int c = 0; c < nc; ++c)
        if (kind[c] == 1) {
            if (!first_ves) first_ves = off[c + 1] - off[c];
            n_slp += off[c + 1] - off[c];
        }
    const int n_dlp = N - n_slp;
    double *x = xmalloc(16 * N), *w = xmalloc(8 * N), *nr = xmalloc(16 * N), *k = xmalloc(8 * N);
    double *s = xmalloc(16 * n_slp), *t = xmalloc(16 * n_dlp);
    int *sel = xmalloc(4 * nsel);
    double *fr = xmalloc(16 * nfree);
    rd(x, 16, N, f); rd(w, 8, N, f); rd(nr, 16, N, f); rd(k, 8, N, f);
    rd(s, 16, n_slp, f); rd(t, 16, n_dlp, f);
    rd(sel, 4, nsel, f); rd(fr, 16, nfree, f);
    fclose(f);
    /* exact-size outputs, so any write past the end is caught */
    double *o_all = xmalloc(16 * N), *o_sel = xmalloc(16 * nsel), *o_free = xmalloc(16 * nfree);
    double *R = xmalloc(8 * (first_ves ? first_ves : 1));
    int st[6];
    st[0] = ora_sum(N, nc, off, kind, x, w, nr, k, par[0], par[1], s, t, par[2], 0, NULL, o_all, 2);
    st[1] = ora_sum(N, nc, off, kind, x, w, nr, k, par[0], par[1], s, t, par[2], nsel, sel, o_sel, 2);
    st[2] = ora_sum_free(N, nc, off, kind, x, w, nr, par[0], par[1], s, t, nfree, fr, o_free, 2);
    st[3] = first_ves ? ora_kress_weights(first_ves, R) : 0;
    /* argument checks: an odd vesicle size and inconsistent offsets must be refused */
    int bad_off[2] = {0, 7}, bad_kind[1] = {1};
    st[4] = ora_sum(7, 1, bad_off, bad_kind, x, w, nr, k, par[0], par[1], s, t, 0.0, 0, NULL,
                    o_all, 1);
    int bad_off2[2] = {1, N};
    st[5] = ora_sum(N, 1, bad_off2, kind, x, w, nr, k, par[0], par[1], s, t, 0.0, 0, NULL, o_all, 1);
    FILE *o = fopen(argv[2], "wb");
    if (!o) return 2;
    /* the node sum again for the output: the bad calls above must not have written into it */
    st[0] |= ora_sum(N, nc, off, kind, x, w, nr, k, par[0], par[1], s, t, par[2], 0, NULL, o_all, 2);
    fwrite(o_all, 16, N, o);
    fwrite(o_sel, 16, nsel, o);
    fwrite(o_free, 16, nfree, o);
    if (first_ves) fwrite(R, 8, first_ves, o);
    fwrite(st, 4, 6, o);
    fclose(o);
    free(off); free(kind); free(x); free(w); free(nr); free(k); free(s); free(t); free(sel);
    free(fr); free(o_all); free(o_sel); free(o_free); free(R);
    return (st[0] || st[1] || st[2] || st[3]) ? 1 : 0;
}
