"""FP64 CPU oracle for the FX correlator hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct numpy implementations of what the correlator
computes (polyphase filter bank, channeliser, delay/phase correction,
cross-multiply-accumulate, MAD flagging, requantised correlation and the
learned flagger's conv net).  Only the test-suite, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import this package; the product
path never calls it and shares no code with it.
"""
