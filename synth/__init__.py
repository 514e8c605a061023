"""Seeded synthetic input generators (no clutter-filter arithmetic here)."""
from .iq import (Recipe, SMALL_96x64x32, REALTIME_256x128x100, STREAM_512x256x200,  # noqa: F401
                 STRESS_256x192x300, LEARNED_384x256x128, generate_packet, generate_frames,
                 packet_ring)
