"""TEST INFRASTRUCTURE — the CPU oracle of pixel local reconstruction (see oracle.py)."""
