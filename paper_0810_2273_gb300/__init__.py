"""GB300-native vdW-DF nonlocal correlation (JuNoLo hot path), placeholder."""
