"""GB300-native vortex-particle hot path of the NL-UVLM-VPM method (arXiv 2511.11430)."""
