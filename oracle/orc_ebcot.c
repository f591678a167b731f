/*
 * FlowRoI oracle, part 2: embedded block coding of the RoI-shifted
 * coefficients (plain C, test infrastructure only; see flowroi_oracle.c).
 *
 * The paper codes its frames with an off-the-shelf JPEG2000 encoder under
 * scaling-based RoI (§Implementation details, Table 1: the RoI coefficients
 * are scaled up by the user's scaling factor, then the codestream is cut to
 * the target compression rate).  This file is that coder's embedded block
 * coder, written from the JPEG2000 Part 1 definitions (ISO/IEC 15444-1):
 *
 *   - MQ arithmetic coder (Annex C): 47-state probability table, 19
 *     contexts, encoder INITENC / ENCODE / FLUSH, decoder INITDEC / DECODE;
 *   - bit-plane coding passes of a code-block (Annex D): stripes of four
 *     rows; significance propagation, magnitude refinement and cleanup
 *     (with run-length mode); zero-coding contexts by sub-band orientation,
 *     sign-coding contexts with the sign-flip bit, refinement contexts;
 *   - every pass terminated (the "termination on each coding pass" mode),
 *     so each pass is its own byte segment and a truncation point;
 *   - per pass, the decrease of the squared error of the midpoint
 *     reconstruction (in doubled units, so every term is an integer);
 *   - rate control (post-compression rate-distortion optimisation, Annex
 *     J): the lower convex hull of each code-block's (bytes, distortion
 *     decrease) truncation points here; the slope threshold that fits a
 *     byte budget is found in oracle.py.
 *
 * Readings where the definitions leave the choice to the encoder: every
 * pass terminated with the standard FLUSH; contexts keep their states
 * across passes of a code-block; code-blocks 64 x 64 anchored at each
 * sub-band's origin; distortion measured on the quantised (RoI-shifted)
 * coefficients with unit band weights: the 9/7 steps are already energy
 * weighted (equal steps cost equal image-domain error), and the RoI shift
 * makes RoI errors count 2^(2s) times, which is the priority scaling-based
 * RoI asks for.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ----------------------------------------------------- MQ coder (Annex C) */

typedef struct {
    uint16_t qe;
    uint8_t nmps, nlps, sw;
} orc_mq_state;

static const orc_mq_state MQ[47] = {
    {0x5601, 1, 1, 1},   {0x3401, 2, 6, 0},   {0x1801, 3, 9, 0},   {0x0AC1, 4, 12, 0},  {0x0521, 5, 29, 0},
    {0x0221, 38, 33, 0}, {0x5601, 7, 6, 1},   {0x5401, 8, 14, 0},  {0x4801, 9, 14, 0},  {0x3801, 10, 14, 0},
    {0x3001, 11, 17, 0}, {0x2401, 12, 18, 0}, {0x1C01, 13, 20, 0}, {0x1601, 29, 21, 0}, {0x5601, 15, 14, 1},
    {0x5401, 16, 14, 0}, {0x5101, 17, 15, 0}, {0x4801, 18, 16, 0}, {0x3801, 19, 17, 0}, {0x3401, 20, 18, 0},
    {0x3001, 21, 19, 0}, {0x2801, 22, 19, 0}, {0x2401, 23, 20, 0}, {0x2201, 24, 21, 0}, {0x1C01, 25, 22, 0},
    {0x1801, 26, 23, 0}, {0x1601, 27, 24, 0}, {0x1401, 28, 25, 0}, {0x1201, 29, 26, 0}, {0x1101, 30, 27, 0},
    {0x0AC1, 31, 28, 0}, {0x09C1, 32, 29, 0}, {0x08A1, 33, 30, 0}, {0x0521, 34, 31, 0}, {0x0441, 35, 32, 0},
    {0x02A1, 36, 33, 0}, {0x0221, 37, 34, 0}, {0x0141, 38, 35, 0}, {0x0111, 39, 36, 0}, {0x0085, 40, 37, 0},
    {0x0049, 41, 38, 0}, {0x0025, 42, 39, 0}, {0x0015, 43, 40, 0}, {0x0009, 44, 41, 0}, {0x0005, 45, 42, 0},
    {0x0001, 45, 43, 0}, {0x5601, 46, 46, 0},
};

/* The table as plain arrays (for the tests that check its structure). */
int orc_mq_table(int32_t *qe, int32_t *nmps, int32_t *nlps, int32_t *sw)
{
    for (int i = 0; i < 47; i++) {
        qe[i] = MQ[i].qe;
        nmps[i] = MQ[i].nmps;
        nlps[i] = MQ[i].nlps;
        sw[i] = MQ[i].sw;
    }
    return 47;
}

enum { CTX_ZC = 0, CTX_SC = 9, CTX_MR = 14, CTX_RL = 17, CTX_UNI = 18, NCTX = 19 };

/* context states: index into MQ and the more probable symbol */
typedef struct {
    uint8_t i[NCTX], mps[NCTX];
} orc_ctx;

static void ctx_reset(orc_ctx *c)
{
    for (int k = 0; k < NCTX; k++) c->i[k] = 0, c->mps[k] = 0;
    c->i[CTX_ZC] = 4;
    c->i[CTX_RL] = 3;
    c->i[CTX_UNI] = 46;
}

typedef struct {
    uint32_t a, c;
    int ct;
    uint8_t *buf; /* buf[-1] is a scratch byte */
    long bp;      /* index of the current byte B (starts at -1) */
} orc_mqe;

static void mqe_init(orc_mqe *e, uint8_t *buf)
{
    e->a = 0x8000;
    e->c = 0;
    e->ct = 12;
    e->buf = buf;
    e->bp = -1;
    e->buf[-1] = 0;
}

static void mqe_byteout(orc_mqe *e)
{
    if (e->buf[e->bp] == 0xFF) {
        e->bp++;
        e->buf[e->bp] = (uint8_t)(e->c >> 20);
        e->c &= 0xFFFFF;
        e->ct = 7;
    } else if (e->c < 0x8000000) {
        e->bp++;
        e->buf[e->bp] = (uint8_t)(e->c >> 19);
        e->c &= 0x7FFFF;
        e->ct = 8;
    } else {
        e->buf[e->bp]++;
        if (e->buf[e->bp] == 0xFF) {
            e->c &= 0x7FFFFFF;
            e->bp++;
            e->buf[e->bp] = (uint8_t)(e->c >> 20);
            e->c &= 0xFFFFF;
            e->ct = 7;
        } else {
            e->bp++;
            e->buf[e->bp] = (uint8_t)(e->c >> 19);
            e->c &= 0x7FFFF;
            e->ct = 8;
        }
    }
}

static void mqe_renorm(orc_mqe *e)
{
    do {
        e->a <<= 1;
        e->c <<= 1;
        e->ct--;
        if (e->ct == 0) mqe_byteout(e);
    } while ((e->a & 0x8000) == 0);
}

static void mqe_encode(orc_mqe *e, orc_ctx *x, int cx, int d)
{
    const orc_mq_state *s = &MQ[x->i[cx]];
    const uint32_t qe = s->qe;
    e->a -= qe;
    if (d == x->mps[cx]) {
        if ((e->a & 0x8000) == 0) {
            if (e->a < qe) e->a = qe;
            else e->c += qe;
            x->i[cx] = s->nmps;
            mqe_renorm(e);
        } else {
            e->c += qe;
        }
    } else {
        if (e->a < qe) e->c += qe;
        else e->a = qe;
        if (s->sw) x->mps[cx] ^= 1;
        x->i[cx] = s->nlps;
        mqe_renorm(e);
    }
}

/* Terminates the codeword; returns the segment length in bytes. */
static long mqe_flush(orc_mqe *e)
{
    const uint32_t tempc = e->c + e->a;
    e->c |= 0xFFFF;
    if (e->c >= tempc) e->c -= 0x8000;
    e->c <<= e->ct;
    mqe_byteout(e);
    e->c <<= e->ct;
    mqe_byteout(e);
    if (e->buf[e->bp] != 0xFF) e->bp++;
    return e->bp;
}

typedef struct {
    uint32_t a, c;
    int ct;
    const uint8_t *buf;
    long n, bp;
} orc_mqd;

static uint8_t mqd_at(const orc_mqd *d, long i) { return i < d->n ? d->buf[i] : 0xFF; }

static void mqd_bytein(orc_mqd *d)
{
    if (mqd_at(d, d->bp) == 0xFF) {
        if (mqd_at(d, d->bp + 1) > 0x8F) {
            d->c += 0xFF00;
            d->ct = 8;
        } else {
            d->bp++;
            d->c += (uint32_t)mqd_at(d, d->bp) << 9;
            d->ct = 7;
        }
    } else {
        d->bp++;
        d->c += (uint32_t)mqd_at(d, d->bp) << 8;
        d->ct = 8;
    }
}

static void mqd_init(orc_mqd *d, const uint8_t *buf, long n)
{
    d->buf = buf;
    d->n = n;
    d->bp = 0;
    d->c = (uint32_t)mqd_at(d, 0) << 16;
    mqd_bytein(d);
    d->c <<= 7;
    d->ct -= 7;
    d->a = 0x8000;
}

static void mqd_renorm(orc_mqd *d)
{
    do {
        if (d->ct == 0) mqd_bytein(d);
        d->a <<= 1;
        d->c <<= 1;
        d->ct--;
    } while ((d->a & 0x8000) == 0);
}

static int mqd_decode(orc_mqd *d, orc_ctx *x, int cx)
{
    const orc_mq_state *s = &MQ[x->i[cx]];
    const uint32_t qe = s->qe;
    int out;
    d->a -= qe;
    if ((d->c >> 16) < qe) {
        /* LPS exchange */
        if (d->a < qe) {
            d->a = qe;
            out = x->mps[cx];
            x->i[cx] = s->nmps;
        } else {
            d->a = qe;
            out = 1 - x->mps[cx];
            if (s->sw) x->mps[cx] ^= 1;
            x->i[cx] = s->nlps;
        }
        mqd_renorm(d);
    } else {
        d->c -= qe << 16;
        if ((d->a & 0x8000) == 0) {
            /* MPS exchange */
            if (d->a < qe) {
                out = 1 - x->mps[cx];
                if (s->sw) x->mps[cx] ^= 1;
                x->i[cx] = s->nlps;
            } else {
                out = x->mps[cx];
                x->i[cx] = s->nmps;
            }
            mqd_renorm(d);
        } else {
            out = x->mps[cx];
        }
    }
    return out;
}

/* MQ round trip on a decision sequence: encodes n decisions d[] in
 * contexts cx[] (one terminated codeword), returns its length; the
 * decoder's decisions go to out[].  The context states start as a
 * code-block's do. */
long orc_mq_roundtrip(const uint8_t *d, const uint8_t *cx, long n, uint8_t *code, uint8_t *out)
{
    orc_ctx xe, xd;
    ctx_reset(&xe);
    ctx_reset(&xd);
    orc_mqe e;
    mqe_init(&e, code + 1);
    for (long k = 0; k < n; k++) mqe_encode(&e, &xe, cx[k], d[k]);
    const long len = mqe_flush(&e);
    memmove(code, code + 1, (size_t)len);
    orc_mqd dd;
    mqd_init(&dd, code, len);
    for (long k = 0; k < n; k++) out[k] = (uint8_t)mqd_decode(&dd, &xd, cx[k]);
    return len;
}

/* ---------------------------------------------- coding passes (Annex D) */

/* Sub-band orientations of the zero-coding table. */
enum { ORI_LL = 0, ORI_HL = 1, ORI_LH = 2, ORI_HH = 3 };

/* Zero-coding context from the significant horizontal (h, 0..2), vertical
 * (v, 0..2) and diagonal (d, 0..4) neighbours. */
static int zc_context(int ori, int h, int v, int d)
{
    if (ori == ORI_HL) {
        const int t = h;
        h = v;
        v = t;
    }
    if (ori != ORI_HH) {
        if (h == 2) return 8;
        if (h == 1) return v >= 1 ? 7 : (d >= 1 ? 6 : 5);
        if (v == 2) return 4;
        if (v == 1) return 3;
        return d >= 2 ? 2 : (d == 1 ? 1 : 0);
    }
    const int hv = h + v;
    if (d >= 3) return 8;
    if (d == 2) return hv >= 1 ? 7 : 6;
    if (d == 1) return hv >= 2 ? 5 : (hv == 1 ? 4 : 3);
    return hv >= 2 ? 2 : (hv == 1 ? 1 : 0);
}

/* Sign-coding context (9..13) and sign-flip bit from the horizontal and
 * vertical contributions (each clipped to -1..1). */
static void sc_context(int hc, int vc, int *cx, int *flip)
{
    if (hc < 0) {
        hc = -hc;
        vc = -vc;
        *flip = 1;
    } else if (hc == 0 && vc < 0) {
        vc = -vc;
        *flip = 1;
    } else {
        *flip = 0;
    }
    if (hc == 1) *cx = vc == 1 ? 13 : (vc == 0 ? 12 : 11);
    else *cx = vc == 1 ? 10 : 9;
}

/* The context rules as tables (for the tests that check their structure):
 * zc[ori * 45 + h + 3 v + 9 d], and sc / flip at (hc + 1) + 3 (vc + 1). */
void orc_context_tables(int32_t *zc, int32_t *sc, int32_t *flip)
{
    for (int o = 0; o < 4; o++)
        for (int d = 0; d < 5; d++)
            for (int v = 0; v < 3; v++)
                for (int h = 0; h < 3; h++) zc[o * 45 + h + 3 * v + 9 * d] = zc_context(o, h, v, d);
    for (int vc = -1; vc <= 1; vc++)
        for (int hc = -1; hc <= 1; hc++) {
            int cx = 0, fl = 0;
            sc_context(hc, vc, &cx, &fl);
            sc[(hc + 1) + 3 * (vc + 1)] = cx;
            flip[(hc + 1) + 3 * (vc + 1)] = fl;
        }
}

/* Code-block coder state: magnitudes, signs and flags with a one-sample
 * border of zeros (neighbours outside the code-block are insignificant). */
#define CB_MAX 64
#define CB_S (CB_MAX + 2)
enum { F_SIG = 1, F_REF = 2, F_VIS = 4, F_NEG = 8 };

typedef struct {
    int w, h, ori;
    uint8_t f[CB_S * CB_S];
    uint8_t kp[CB_S * CB_S]; /* decoder: lowest plane whose bit is known */
    uint32_t m[CB_S * CB_S];
} orc_cb;

static inline int cbi(int x, int y) { return (y + 1) * CB_S + (x + 1); }

static void nb_counts(const orc_cb *b, int x, int y, int *h, int *v, int *d)
{
    const uint8_t *f = b->f;
    const int i = cbi(x, y);
    *h = (f[i - 1] & F_SIG) + (f[i + 1] & F_SIG);
    *v = (f[i - CB_S] & F_SIG) + (f[i + CB_S] & F_SIG);
    *d = (f[i - CB_S - 1] & F_SIG) + (f[i - CB_S + 1] & F_SIG) + (f[i + CB_S - 1] & F_SIG) + (f[i + CB_S + 1] & F_SIG);
}

static int contrib(uint8_t a, uint8_t b)
{
    int s = 0;
    if (a & F_SIG) s += (a & F_NEG) ? -1 : 1;
    if (b & F_SIG) s += (b & F_NEG) ? -1 : 1;
    return s < -1 ? -1 : (s > 1 ? 1 : s);
}

static void sign_ctx(const orc_cb *b, int x, int y, int *cx, int *flip)
{
    const int i = cbi(x, y);
    sc_context(contrib(b->f[i - 1], b->f[i + 1]), contrib(b->f[i - CB_S], b->f[i + CB_S]), cx, flip);
}

/* Doubled-unit reconstruction of magnitude m once planes >= p are known:
 * 2 * (m with bits below p cleared) + 2^p (the interval midpoint), or 0
 * while m >> p == 0. */
static int64_t recon2(uint32_t m, int p)
{
    if ((m >> p) == 0) return 0;
    return 2 * (int64_t)((m >> p) << p) + (p > 0 ? ((int64_t)1 << p) : 0);
}

/* Decrease of the squared error (doubled units) when m's reconstruction
 * goes from planes >= p_before known (p_before > 31: not yet significant)
 * to planes >= p_after known.  Exact in int64 for m < 2^24. */
static int64_t derr(uint32_t m, int p_before, int p_after)
{
    const int64_t t = 2 * (int64_t)m;
    const int64_t eb = t - (p_before > 31 ? 0 : recon2(m, p_before));
    const int64_t ea = t - recon2(m, p_after);
    return eb * eb - ea * ea;
}

/* Number of magnitude bit-planes of a code-block (0 when all zero). */
static int cb_planes(const orc_cb *b)
{
    uint32_t mx = 0;
    for (int y = 0; y < b->h; y++)
        for (int x = 0; x < b->w; x++) mx |= b->m[cbi(x, y)];
    int n = 0;
    while (mx) n++, mx >>= 1;
    return n;
}

static void cb_load(orc_cb *b, const int32_t *q, int stride, int w, int h, int ori)
{
    memset(b, 0, sizeof *b);
    b->w = w;
    b->h = h;
    b->ori = ori;
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            const int32_t v = q[(int64_t)y * stride + x];
            const int i = cbi(x, y);
            b->m[i] = v < 0 ? (uint32_t)(-(int64_t)v) : (uint32_t)v;
            if (v < 0) b->f[i] |= F_NEG;
        }
}

/* Codes (enc) or decodes one pass of plane p.  type 0 = significance
 * propagation, 1 = magnitude refinement, 2 = cleanup.  Decoding sets bits
 * of b->m and the sign flags.  Returns the pass's distortion decrease
 * (encoding only), an exact integer sum (so independent of the order of
 * summation). */
static int64_t cb_pass(orc_cb *b, int type, int p, orc_ctx *x, orc_mqe *e, orc_mqd *dd)
{
    int64_t dd_sum = 0;
    const int enc = e != NULL;
    for (int y0 = 0; y0 < b->h; y0 += 4) {
        const int y1 = y0 + 4 < b->h ? y0 + 4 : b->h;
        for (int cx = 0; cx < b->w; cx++) {
            int y = y0;
            if (type == 2 && y1 - y0 == 4) {
                /* run-length mode: four insignificant, unvisited samples
                 * with all-zero neighbourhoods */
                int rl = 1;
                for (int yy = y0; yy < y1 && rl; yy++) {
                    const int i = cbi(cx, yy);
                    int h, v, d;
                    nb_counts(b, cx, yy, &h, &v, &d);
                    if ((b->f[i] & (F_SIG | F_VIS)) || h + v + d) rl = 0;
                }
                if (rl) {
                    int r = 4;
                    if (enc) {
                        for (int yy = y0; yy < y1; yy++)
                            if ((b->m[cbi(cx, yy)] >> p) & 1) {
                                r = yy - y0;
                                break;
                            }
                        mqe_encode(e, x, CTX_RL, r < 4);
                        if (r == 4) continue;
                        mqe_encode(e, x, CTX_UNI, r >> 1);
                        mqe_encode(e, x, CTX_UNI, r & 1);
                    } else {
                        if (!mqd_decode(dd, x, CTX_RL)) continue;
                        r = mqd_decode(dd, x, CTX_UNI) << 1;
                        r |= mqd_decode(dd, x, CTX_UNI);
                        b->m[cbi(cx, y0 + r)] |= 1u << p;
                        for (int yy = y0; yy <= y0 + r; yy++) b->kp[cbi(cx, yy)] = (uint8_t)p;
                    }
                    /* sample y0 + r is significant: its sign */
                    const int i = cbi(cx, y0 + r);
                    int scx, flip;
                    sign_ctx(b, cx, y0 + r, &scx, &flip);
                    if (enc) {
                        mqe_encode(e, x, scx, ((b->f[i] & F_NEG) ? 1 : 0) ^ flip);
                        dd_sum += derr(b->m[i], 32, p);
                    } else if (mqd_decode(dd, x, scx) ^ flip) {
                        b->f[i] |= F_NEG;
                    }
                    b->f[i] |= F_SIG;
                    y = y0 + r + 1;
                }
            }
            for (; y < y1; y++) {
                const int i = cbi(cx, y);
                uint8_t *fl = &b->f[i];
                int h, v, d;
                nb_counts(b, cx, y, &h, &v, &d);
                if (type == 0) {
                    if ((*fl & F_SIG) || h + v + d == 0) continue;
                } else if (type == 1) {
                    if (!(*fl & F_SIG) || (*fl & F_VIS)) continue;
                    const int mcx = (*fl & F_REF) ? 16 : (h + v + d ? 15 : 14);
                    if (enc) {
                        mqe_encode(e, x, mcx, (b->m[i] >> p) & 1);
                        dd_sum += derr(b->m[i], p + 1, p);
                    } else {
                        if (mqd_decode(dd, x, mcx)) b->m[i] |= 1u << p;
                        b->kp[i] = (uint8_t)p;
                    }
                    *fl |= F_REF;
                    continue;
                } else {
                    if (*fl & (F_SIG | F_VIS)) continue;
                }
                /* zero coding (passes 0 and 2) */
                const int zcx = zc_context(b->ori, h, v, d);
                int bit;
                if (enc) {
                    bit = (b->m[i] >> p) & 1;
                    mqe_encode(e, x, zcx, bit);
                } else {
                    bit = mqd_decode(dd, x, zcx);
                    if (bit) b->m[i] |= 1u << p;
                    b->kp[i] = (uint8_t)p;
                }
                if (type == 0) *fl |= F_VIS;
                if (bit) {
                    int scx, flip;
                    sign_ctx(b, cx, y, &scx, &flip);
                    if (enc) {
                        mqe_encode(e, x, scx, ((*fl & F_NEG) ? 1 : 0) ^ flip);
                        dd_sum += derr(b->m[i], 32, p);
                    } else if (mqd_decode(dd, x, scx) ^ flip) {
                        *fl |= F_NEG;
                    }
                    *fl |= F_SIG;
                }
            }
        }
    }
    if (type == 2)
        for (int y = 0; y < b->h; y++)
            for (int cx = 0; cx < b->w; cx++) b->f[cbi(cx, y)] &= (uint8_t)~F_VIS;
    return dd_sum;
}

/* Encodes one code-block (w, h <= 64) of orientation ori, magnitudes below
 * 2^24.  Writes the passes' segments back to back into out (capacity cap),
 * their lengths to plen[] and distortion decreases (the pass's int64 sum,
 * then converted to double) to dist[]; returns the number of passes (3
 * planes - 2, 0 for an all-zero block) and the planes in *planes, -1 when
 * out is too small, -2 for a magnitude of 2^24 or more.  Every pass is
 * terminated (the code-block style option "termination on each coding
 * pass"); with reset the context states also return to their initial
 * values at the start of every pass (the option "reset context
 * probabilities on coding pass boundaries"), else they carry from pass to
 * pass.  Both options are signalled in the code-block style byte of the
 * COD marker (Annex A.6.1). */
int orc_t1_encode(const int32_t *q, int stride, int w, int h, int ori, uint8_t *out, long cap, int *planes,
                  int32_t *plen, double *dist, int reset)
{
    static orc_cb b;
    cb_load(&b, q, stride, w, h, ori);
    const int mb = cb_planes(&b);
    *planes = mb;
    if (mb == 0) return 0;
    if (mb > 24) return -2;
    orc_ctx x;
    ctx_reset(&x);
    /* scratch: one byte before each segment for the coder's B register, and
     * slack after it for the flush */
    uint8_t *tmp = (uint8_t *)malloc((size_t)(8 * 64 * 64 + 64));
    long pos = 0;
    int k = 0;
    for (int p = mb - 1; p >= 0; p--) {
        for (int type = (p == mb - 1 ? 2 : 0); type <= 2; type++, k++) {
            orc_mqe e;
            mqe_init(&e, tmp + 1);
            if (reset) ctx_reset(&x);
            dist[k] = (double)cb_pass(&b, type, p, &x, &e, NULL);
            const long len = mqe_flush(&e);
            if (pos + len > cap) {
                free(tmp);
                return -1;
            }
            memcpy(out + pos, tmp + 1, (size_t)len);
            plen[k] = (int32_t)len;
            pos += len;
        }
    }
    free(tmp);
    return k;
}

/* Decodes the first nkept passes of a code-block coded by orc_t1_encode
 * (segments back to back in code, lengths plen[]) into q.  With midpoint,
 * a significant coefficient whose bits are known down to plane p is set to
 * the middle of its interval (the known bits plus 2^(p-1), p > 0): the
 * reconstruction whose squared error the encoder's distortion decreases
 * account for; without it, to the known bits.  reset: the block was coded
 * with the contexts reset at every pass. */
void orc_t1_decode(const uint8_t *code, const int32_t *plen, int nkept, int planes, int w, int h, int ori,
                   int midpoint, int32_t *q, int stride, int reset)
{
    static orc_cb b;
    memset(&b, 0, sizeof b);
    b.w = w;
    b.h = h;
    b.ori = ori;
    memset(b.kp, planes, sizeof b.kp);
    orc_ctx x;
    ctx_reset(&x);
    long pos = 0;
    int k = 0;
    for (int p = planes - 1; p >= 0 && k < nkept; p--) {
        for (int type = (p == planes - 1 ? 2 : 0); type <= 2 && k < nkept; type++, k++) {
            orc_mqd d;
            mqd_init(&d, code + pos, plen[k]);
            if (reset) ctx_reset(&x);
            cb_pass(&b, type, p, &x, NULL, &d);
            pos += plen[k];
        }
    }
    for (int y = 0; y < h; y++)
        for (int cx = 0; cx < w; cx++) {
            const int i = cbi(cx, y);
            int64_t m = b.m[i];
            if (midpoint && m && b.kp[i] > 0) m += (int64_t)1 << (b.kp[i] - 1);
            q[(int64_t)y * stride + cx] = (int32_t)((b.f[i] & F_NEG) ? -m : m);
        }
}

/* ------------------------------------- rate control (Annex J, PCRD-opt) */

/* Lower convex hull of a code-block's truncation points (bytes R_k,
 * distortion decrease D_k, k = 0..n with R_0 = D_0 = 0, both cumulative):
 * writes the hull's pass counts to hk[] (hk[0] = 0) and the slopes of its
 * segments to hs[] (hs[j] for the segment ending at hk[j], strictly
 * decreasing); returns the number of hull points. */
int orc_hull(int n, const int64_t *R, const double *D, int32_t *hk, double *hs)
{
    int m = 1;
    hk[0] = 0;
    hs[0] = 0.0;
    for (int k = 1; k <= n; k++) {
        if (!(D[k] > D[hk[m - 1]])) continue;
        for (;;) {
            const int a = hk[m - 1];
            const double s = (D[k] - D[a]) / (double)(R[k] - R[a]);
            if (m >= 2 && s >= hs[m - 1]) {
                m--; /* hk[m] is not on the hull */
                continue;
            }
            hk[m] = k;
            hs[m] = s;
            m++;
            break;
        }
    }
    return m;
}
