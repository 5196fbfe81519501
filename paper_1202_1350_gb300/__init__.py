"""GB300 prover and verifier for the GKR/CMT interactive proof over F_p,
p = 2^61 - 1 (Thaler, Roberts, Mitzenmacher, Pfister, "Verifiable Computation
with Massively Parallel Interactive Proofs").

The compute path is the CUDA library built from ``csrc/`` (``libvc.so``); this
package only marshals arguments to its C ABI (``include/vc.h``).  Importing the
package does not load the library; the first call does, and fails loudly if it
has not been built.
"""
from .vc import (EXPLICIT, F0_FINAL, F0_FIRST, F0_PAIR, MATMULT, P, SQUARE, TREE, VcError,  # noqa: F401
                 vc_circuit_bytes, vc_circuit_create, vc_circuit_get_info, vc_circuit_set_stage_events, vc_circuit_destroy, vc_circuit_sync, vc_evaluate,
                 vc_field_mul, vc_field_mul_rate, vc_prove, vc_prove_batch, vc_status_string,
                 vc_transcript_len, vc_verify)
from .api import Batch, Circuit, Server  # noqa: F401
