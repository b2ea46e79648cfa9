"""Seeded synthetic baseband streams for the FX correlator.

This package only draws input samples (noise, a delayed common source, RFI
tones, chirps and bursts) and rounds them to int8.  It contains none of the
correlator's own arithmetic (no polyphase filter, channeliser, correlator or
flagger), so both the FP64 oracle and the CUDA path can take their inputs from
it without sharing any of the method's code.
"""

from .streams import (  # noqa: F401
    StreamSpec,
    make_stream,
    make_stream_iq,
    config_c1,
    config_c2,
    config_c3,
    config_c4_streams,
    delays_for,
)
