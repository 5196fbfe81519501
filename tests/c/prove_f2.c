/* A C user of include/vc.h: builds the F2 circuit for 2^n inputs
 * x_i = (i * 2654435761) mod 65537, proves it with host buffers on device 0,
 * verifies the proof, proves and verifies it again in one call, and prints
 * the statuses, the accept bits and the transcript (one decimal u64 per
 * line).  Usage: prove_f2 n seed */
#include <inttypes.h>
#include <stdio.h>
#include <stdlib.h>

#include "vc.h"

int main(int argc, char **argv)
{
    if (argc != 3) {
        fprintf(stderr, "usage: %s n seed\n", argv[0]);
        return 2;
    }
    const uint32_t n = (uint32_t)atoi(argv[1]);
    const uint64_t seed = strtoull(argv[2], NULL, 10);
    if (n > 24) return 2;
    /* layers 0..n: the addition tree (width 2^i), layer n: squares, layer n+1: inputs */
    uint32_t log_width[26], wiring[25];
    for (uint32_t i = 0; i <= n; i++) log_width[i] = i;
    log_width[n + 1] = n;
    for (uint32_t i = 0; i < n; i++) wiring[i] = VC_WIRE_TREE;
    wiring[n] = VC_WIRE_SQUARE;
    vc_circuit_desc desc = {n + 1, log_width, wiring, NULL, NULL, NULL};

    vc_circuit *c = NULL;
    vc_status st = vc_circuit_create(&desc, 0, &c);
    if (st != VC_OK) {
        printf("create %s\n", vc_status_string(st));
        return 1;
    }
    uint64_t len = 0;
    vc_transcript_len(c, &len);
    const uint64_t nin = (uint64_t)1 << n;
    uint64_t *x = malloc(nin * sizeof(uint64_t)), *tr = malloc(len * sizeof(uint64_t));
    if (!x || !tr) return 1;
    for (uint64_t i = 0; i < nin; i++) x[i] = (i * 2654435761ull) % 65537ull;

    st = vc_prove(c, x, seed, tr, NULL);  /* host buffers: returns once tr is written */
    printf("prove %s\n", vc_status_string(st));
    int accept = -1;
    st = vc_verify(c, x, seed, tr, &accept, NULL);
    printf("verify %s %d\n", vc_status_string(st), accept);
    tr[len - 1] += 1; /* a changed last entry must be rejected */
    int reject = -1;
    vc_verify(c, x, seed, tr, &reject, NULL);
    tr[len - 1] -= 1;
    printf("tampered %d\n", reject);
    /* the same proof and its verification in one call */
    uint64_t *tr2 = malloc(len * sizeof(uint64_t));
    if (!tr2) return 1;
    int accept2 = -1;
    st = vc_prove_verify(c, x, seed, tr2, &accept2, NULL);
    int same = 1;
    for (uint64_t k = 0; k < len; k++) same &= tr2[k] == tr[k];
    printf("prove_verify %s %d %d\n", vc_status_string(st), accept2, same);
    free(tr2);
    for (uint64_t k = 0; k < len; k++) printf("%" PRIu64 "\n", tr[k]);
    vc_circuit_destroy(c);
    free(x);
    free(tr);
    return 0;
}
